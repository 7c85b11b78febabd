"""Reporting logic of bench.py on CPU: the roofline object (dominant kernel,
algorithmic bytes or FLOPs per launch, bound, fraction of the peak) and the
source-hash check that keeps recorded ncu traffic only for the kernel code it
was measured on."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Inst:
    def __init__(self, dims):
        self.dims = dims
        self.n = 1
        for d in dims:
            self.n *= d


def test_roofline_mixed_is_hbm_bound():
    import bench
    peak, _ = bench.measured_peaks()
    inst = _Inst((2048, 2048))
    # kernel -> (avg ms per timed launch, timed launches, total ms)
    res = {"kernel_ms": {"mixed_cg_init": (0.03, 10, 0.3), "mixed_cg": (0.04, 10, 0.4),
                         "mixed_residual64": (0.4, 1, 0.4)}}
    r = bench.roofline(res, inst, "c2")
    assert r["bound"] == "hbm" and r["kernel"] == "mixed_cg" and r["unit"] == "GB/s"
    algo = 28 * inst.n
    assert r["algorithmic_bytes_per_launch"] == algo
    assert r["achieved"] == pytest.approx(algo / 0.04e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, abs=2e-4)
    assert r["share_of_kernel_time"] == pytest.approx(0.4 / 1.1, abs=1e-3)


@pytest.mark.parametrize("dims,bytes_per_node", [((2048, 2048), 95), ((256, 256, 256), 85)])
def test_multigrid_iteration_roofline_is_separate(dims, bytes_per_node):
    """The multigrid-preconditioned iteration (all its kernels, timed as one
    unit) never becomes the dominant kernel of a Jacobi line; asked for by
    name it reports its own per-dimension algorithmic bytes."""
    import bench
    inst = _Inst(dims)
    res = {"kernel_ms": {"mixed_mg": (0.3, 90, 27.0), "mixed_cg": (0.04, 10, 0.4),
                         "mixed_residual64": (0.4, 1, 0.4)}}
    r = bench.roofline(res, inst, "c2")
    assert r["kernel"] == "mixed_cg"
    m = bench.roofline(res, inst, "c2", only="mixed_mg")
    assert m["kernel"] == "mixed_mg" and m["bound"] == "hbm"
    assert m["algorithmic_bytes_per_launch"] == bytes_per_node * inst.n
    assert m["achieved"] == pytest.approx(bytes_per_node * inst.n / 0.3e-3 / 1e9, rel=1e-3)
    assert bench.algo_bytes("mixed_mg", inst) == bytes_per_node
    assert bench.algo_bytes("mixed_cg", inst) == 28


@pytest.mark.parametrize("dims,flops", [((2048, 2048), 10), ((64, 64, 64), 12)])
def test_roofline_fp64_is_bound_by_the_fp64_rate(dims, flops):
    import bench
    inst = _Inst(dims)
    res = {"kernel_ms": {"cg_pass1_64": (0.08, 5, 0.4), "cg_pass2_64": (0.05, 5, 0.25)}}
    r = bench.roofline(res, inst, "c2")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["kernel"] == "cg_pass1_64"
    assert r["algorithmic_flops_per_launch"] == flops * inst.n
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS, abs=2e-4)


def test_kernel_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    import bench
    csrc = tmp_path / "paper_1403_1937_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// note\n__global__ void k(int *a) { a[0] = 1; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash(["k.cu"])
    (csrc / "k.cu").write_text("/* another\n note */\n__global__ void k(int *a) {\n"
                               "  a[0] = 1;  // same code\n}\n")
    assert bench.kernel_source_hash(["k.cu"]) == h0
    (csrc / "k.cu").write_text("__global__ void k(int *a) { a[0] = 2; }\n")
    assert bench.kernel_source_hash(["k.cu"]) != h0


def test_recorded_traffic_matches_the_committed_kernels():
    """Every entry of profiles/traffic.json for the default kernels is keyed
    to the current source, so the bench reports it (not null)."""
    import bench
    for key in ("cg_pass1_64@c2", "cg_pass2_64@c2", "mixed_cg@c2", "mixed_cg@c3",
                "mixed_cg_packed@c4"):
        kernel, wl = key.split("@")
        assert bench.ncu_traffic(kernel, wl) is not None, key
