"""Packed 2D mixed-precision batches: every inner-CG iteration is one launch
over a tile list spanning all instances (Sec. 6 system per instance).

Each instance is checked against the oracle's relative-form direct solve
(S within 1e-6 at componentwise tol 1e-7), across every packed kernel
variant and tile height, on instances whose inner solves end at different
passes, on ragged and tiny grids, and against the per-instance batch path.
The autotuner's choice is cached in the JSON file and reused."""
import json
import os

import numpy as np
import pytest

from oracle import fd
from paper_1403_1937_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

S_ABS = 1e-6


@pytest.fixture(scope="module")
def eik():
    import torch
    from paper_1403_1937_gb300 import build
    build.build()
    from paper_1403_1937_gb300 import eik as e
    assert torch.cuda.is_available()
    return e


@pytest.fixture(autouse=True)
def no_tune_file(monkeypatch):
    monkeypatch.setenv("EIK_TUNE_CACHE", "off")


def oracle_S(inst):
    sys = fd.assemble(inst.f, inst.dims, inst.h, inst.hbar, inst.src_idx)
    return fd.solve_relative(sys)


def ragged(count, seed, side=(3, 300)):
    """Instances of independent random extents (odd widths, widths below and
    above one 128-column tile, a few rows), 1-4 sources, hbar in {2,4,8} h."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx, ny = (int(v) for v in rng.integers(side[0], side[1] + 1, size=2))
        h = 1.0 / (max(nx, ny) - 1)
        f = wl.fourier_field(rng, (nx, ny), h)
        src = wl.random_sources(rng, nx * ny, int(rng.integers(1, 5)))
        hbar = float(rng.choice([2, 4, 8])) * h
        out.append(wl.Instance((nx, ny), h, hbar, f, src, np.zeros(len(src))))
    return out


def solve_packed(eik, insts, **kw):
    opt = eik.make_options(precision="mixed", tol=1e-7, **kw)
    b = eik.eik_create_batch(insts, opt)
    S, stats = eik.eik_solve_batch(b)
    info = eik.eik_batch_info(b)
    parts = [p.ravel() for p in b.split(S.cpu().numpy())]
    eik.eik_destroy_batch(b)
    return parts, stats, info


@pytest.mark.parametrize("variant,rows", [(1, 8), (2, 16), (3, 5), (4, 32), (1, 13)])
def test_packed_variants_vs_oracle(eik, variant, rows):
    insts = ragged(10, 7 + variant)
    parts, stats, info = solve_packed(eik, insts, tile_override=variant,
                                      batch_tile_rows=rows)
    assert info["packed"] and info["variant"] == variant and info["tile_rows"] == rows
    assert info["tuned"] == "fixed" and info["passes"] > 0
    assert info["node_passes"] > 0 and info["pass_ms"] > 0
    for inst, Si, st in zip(insts, parts, stats):
        assert st["res_cw"] <= 1e-7
        assert np.max(np.abs(Si - oracle_S(inst))) <= S_ABS, inst.dims


def test_packed_matches_per_instance_path(eik):
    """The same batch solved packed and per instance: both meet the oracle
    bound, and they agree with each other to the same order."""
    insts = wl.config4(count=8, side=(48, 260))
    packed, st_p, info = solve_packed(eik, insts, tile_override=1, batch_tile_rows=16)
    single, st_s, info_s = solve_packed(eik, insts, batch_pack=-1)
    assert info["packed"] and not info_s["packed"]
    for inst, a, b in zip(insts, packed, single):
        ref = oracle_S(inst)
        assert np.max(np.abs(a - ref)) <= S_ABS
        assert np.max(np.abs(b - ref)) <= S_ABS
        assert np.max(np.abs(a - b)) <= 2 * S_ABS


def test_packed_tiny_and_single_tile_instances(eik):
    """Instances with one unknown, a 2-row strip, exactly one 128 x 8 tile,
    one column past a tile, next to large ones in the same atlas."""
    def inst(nx, ny, src, hb=4):
        h = 1.0 / (max(nx, ny) - 1)
        rng = np.random.default_rng(nx * 1000 + ny)
        f = wl.fourier_field(rng, (nx, ny), h)
        src = np.array(src, dtype=np.int64)
        return wl.Instance((nx, ny), h, hb * h, f, src, np.zeros(len(src)))
    insts = [inst(2, 2, [0, 1, 2]), inst(65, 2, [0, 64]), inst(128, 8, [5]),
             inst(129, 9, [128 + 129 * 8]), inst(300, 220, [777, 30000], 2),
             inst(3, 3, [0, 2, 6, 8]), inst(257, 31, [100], 8)]
    parts, stats, _ = solve_packed(eik, insts, tile_override=1, batch_tile_rows=8)
    for k, (i, Si) in enumerate(zip(insts, parts)):
        assert np.max(np.abs(Si - oracle_S(i))) <= S_ABS, k


def test_packed_instances_end_at_different_passes(eik):
    """Small and large instances in one batch: the small ones' inner solves
    end many passes before the large ones' (they leave the tile list), and
    both are right."""
    small = ragged(6, 99, side=(8, 24))
    large = ragged(2, 100, side=(380, 420))
    insts = small + large
    parts, stats, info = solve_packed(eik, insts, tile_override=2, batch_tile_rows=8)
    iters = [s["inner_iters"] for s in stats]
    assert max(iters[:6]) * 4 < min(iters[6:])
    for inst, Si in zip(insts, parts):
        assert np.max(np.abs(Si - oracle_S(inst))) <= S_ABS


def test_packed_autotuner_cache(eik, tmp_path, monkeypatch):
    """The first solve of a batch times the candidate tile shapes and writes
    the winner to the cache file under (GPU, 2d-mixed, size class); a second
    batch of the same size class reads it."""
    path = tmp_path / "tune.json"
    monkeypatch.setenv("EIK_TUNE_CACHE", str(path))
    insts = ragged(6, 5, side=(40, 200))
    parts, _, info = solve_packed(eik, insts)
    assert info["tuned"] == "measured" and 1 <= info["variant"] <= 4
    assert info["tile_rows"] in (8, 16, 32)
    cache = json.loads(path.read_text())
    (key, ent), = cache.items()
    assert "|2d-mixed|" in key
    assert (ent["variant"], ent["ty"]) == (info["variant"], info["tile_rows"])
    assert ent["us_per_pass"] > 0
    parts2, _, info2 = solve_packed(eik, insts)
    assert info2["tuned"] == "cached"
    assert (info2["variant"], info2["tile_rows"]) == (info["variant"], info["tile_rows"])
    for inst, a, b in zip(insts, parts, parts2):
        ref = oracle_S(inst)
        assert np.max(np.abs(a - ref)) <= S_ABS and np.max(np.abs(b - ref)) <= S_ABS


def test_packed_repeated_solves_and_new_f(eik):
    """A packed batch solved twice, then with new f: results follow f."""
    import torch
    insts = ragged(5, 21, side=(30, 150))
    opt = eik.make_options(precision="mixed", tol=1e-7, tile_override=4, batch_tile_rows=16)
    b = eik.eik_create_batch(insts, opt)
    S1, _ = eik.eik_solve_batch(b)
    S2, _ = eik.eik_solve_batch(b)
    assert np.array_equal(S1.cpu().numpy(), S2.cpu().numpy())
    rng = np.random.default_rng(3)
    for i in insts:
        i.f = wl.fourier_field(rng, i.dims, i.h)
    eik.eik_set_f_batch(b, torch.from_numpy(np.concatenate([i.f.ravel() for i in insts])).cuda())
    S3, _ = eik.eik_solve_batch(b)
    for inst, Si in zip(insts, b.split(S3.cpu().numpy())):
        assert np.max(np.abs(Si.ravel() - oracle_S(inst))) <= S_ABS
    eik.eik_destroy_batch(b)


def test_packed_timeout_path(eik):
    """Test hook (eik_options.test_flags bit 0): in the first pass one warp
    never gets its first row copy, its bounded wait (0.2 s) expires, the pass
    flags the fault, the executor abandons the solve and every instance
    returns EIK_ERR_TIMEOUT; no GPU fault is involved.  A batch created
    without the hook then solves normally."""
    from paper_1403_1937_gb300 import _lib
    insts = ragged(4, 31, side=(40, 160))
    opt = eik.make_options(precision="mixed", tol=1e-7, tile_override=1, batch_tile_rows=16,
                           test_flags=1)
    b = eik.eik_create_batch(insts, opt)
    with pytest.raises(_lib.EikError) as ei:
        eik.eik_solve_batch(b)
    assert ei.value.status == _lib.EIK_ERR_TIMEOUT
    eik.eik_destroy_batch(b)
    parts, _, _ = solve_packed(eik, insts, tile_override=1, batch_tile_rows=16)
    for inst, Si in zip(insts, parts):
        assert np.max(np.abs(Si - oracle_S(inst))) <= S_ABS
