// Packed 2D mixed-precision batches: atlas, the executor of the batched inner
// solves, and the tile-shape autotuner.
//
// Each instance of a batch solves its own system (Sec. 6, one per instance)
// with its own refinement program, exactly as a single solve does, on its own
// host thread and stream.  What the batch shares is the inner CG: one pass
// launch per CG iteration advances every instance that is in an inner solve,
// over a tile list spanning their grids (k_cg2d_batch), each with its own
// recurrence scalars and stopping test.  An instance joins the list at the
// next pass boundary (a request in a ring of mapped host memory, read by the
// pass's last warp) and leaves it when its inner solve ends (a record in
// mapped host memory that its thread polls), so instances never wait for
// each other.  An executor thread launches the passes as captured CUDA graphs
// of kGraphPasses launches for as long as any instance iterates or waits.
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "eik_batch.h"

namespace eik {

namespace {

constexpr int kGraphPasses = 32;   // even: the buffer sets alternate
constexpr int kTuneWarm = 2, kTuneTimed = 5;
const int kTuneTy[] = {8, 16, 32, 64};

// Synthetic state for timing tile shapes: r = 1, sigma = 1/4 on every node of
// every instance (an SPD operator), the rest as left by creation (zero).
__global__ void k_tune_fill(int64_t total, int P, const int *__restrict__ row_inst,
                            const BInst *__restrict__ bi, float *__restrict__ r0,
                            float *__restrict__ s32) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / P), col = (int)(e % P);
    const int i = row_inst[row];
    if (i >= 0 && col < bi[i].nx) {
      r0[e] = 1.f;
      s32[e] = 0.25f;
    }
  }
}

}  // namespace

struct BatchExec {
  int count = 0, num_sms = 0, boundary = 0, device = 0;
  int variant_req = 0, ty_req = 0;
  std::vector<BInst> h_bi;
  std::vector<int> cells;          // cell count per instance (for the tuner)
  std::vector<int> seq;            // request numbers per instance
  BInst *bi = nullptr;
  MixCtl *st = nullptr;
  int *act = nullptr, *pre = nullptr, *row_inst = nullptr, *alive = nullptr;
  unsigned *cnt = nullptr;
  BatchCtl *bc = nullptr, *h_bc = nullptr;
  BatchRing *ring = nullptr, *d_ring = nullptr;   // mapped host memory
  BatchDone *done = nullptr, *d_done = nullptr;   // mapped host memory
  float *arr[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int P = 0, H = 0;
  int64_t nodes = 0;
  double *part = nullptr;
  int part_cap = 0;
  Cg32BatchBuffers bufs{};
  Cg32BatchPlan plan{};
  bool planned = false;
  int how = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t passes = 0;
  int64_t work = 0;                // sum over passes of the nodes they covered
  double pass_ms = 0.0;            // device time of the executor's graphs
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool bi_dirty = true;
  // executor
  std::thread exec;
  std::mutex mu;
  std::condition_variable cv;
  int live = 0;
  int pushed = 0;                  // requests written to the ring
  std::atomic<int> abort{0};
  eik_status exec_status = EIK_OK;
  std::string msg;
};

namespace {

#define BCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      e->msg = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return EIK_ERR_CUDA;                                                         \
    }                                                                              \
  } while (0)

int tiles_of(const BInst &b, int ty) { return b.tiles_x * ((b.ny + ty - 1) / ty); }

// ------------------------------------------------------------ tuner cache
// One JSON object, one entry per line:
//   "<gpu>|2d-mixed|<size class>": {"variant": V, "ty": T, "us_per_pass": U}
std::string cache_path() {
  const char *env = getenv("EIK_TUNE_CACHE");
  if (env) return (env[0] == 0 || strcmp(env, "off") == 0) ? std::string() : std::string(env);
  std::string dir;
  if (const char *x = getenv("XDG_CACHE_HOME"); x && x[0])
    dir = std::string(x) + "/eik";
  else if (const char *hm = getenv("HOME"); hm && hm[0])
    dir = std::string(hm) + "/.cache/eik";
  else
    return std::string();
  // create the directory chain
  for (size_t k = 1; k <= dir.size(); ++k)
    if (k == dir.size() || dir[k] == '/') mkdir(dir.substr(0, k).c_str(), 0755);
  return dir + "/tune.json";
}

struct TuneEntry {
  int variant = 0, ty = 0;
  double us = 0.0;
};

std::map<std::string, TuneEntry> cache_read(const std::string &path) {
  std::map<std::string, TuneEntry> out;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    const size_t a = line.find('"');
    if (a == std::string::npos) continue;
    const size_t b = line.find('"', a + 1);
    if (b == std::string::npos) continue;
    const std::string key = line.substr(a + 1, b - a - 1);
    const size_t v = line.find("\"variant\":", b), t = line.find("\"ty\":", b);
    const size_t u = line.find("\"us_per_pass\":", b);
    if (v == std::string::npos || t == std::string::npos) continue;
    TuneEntry te;
    te.variant = (int)strtol(line.c_str() + v + 10, nullptr, 10);
    te.ty = (int)strtol(line.c_str() + t + 5, nullptr, 10);
    if (u != std::string::npos) te.us = strtod(line.c_str() + u + 14, nullptr);
    if (te.variant >= 1 && te.variant <= 4 && te.ty >= 1 && te.ty <= 1024) out[key] = te;
  }
  return out;
}

void cache_write(const std::string &path, const std::map<std::string, TuneEntry> &m) {
  const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
  {
    std::ofstream o(tmp);
    if (!o) return;
    o << "{\n";
    size_t k = 0;
    for (const auto &kv : m) {
      char buf[160];
      snprintf(buf, sizeof buf, "{\"variant\": %d, \"ty\": %d, \"us_per_pass\": %.3f}",
               kv.second.variant, kv.second.ty, kv.second.us);
      o << " \"" << kv.first << "\": " << buf << (++k < m.size() ? "," : "") << "\n";
    }
    o << "}\n";
  }
  rename(tmp.c_str(), path.c_str());
}

// Key of the batch: GPU name, dimension and precision, and its size class
// (log2 of the total node count and of the instance count, rounded).
std::string tune_key(const BatchExec *e) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  std::string name = "unknown-gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char &ch : name)
    if (ch == '"' || ch == '|' || ch == '\\') ch = '_';
  char buf[96];
  snprintf(buf, sizeof buf, "|2d-mixed|n2^%d-c2^%d", (int)std::lround(std::log2((double)e->nodes)),
           (int)std::lround(std::log2((double)e->count)));
  return name + buf;
}

// Uploads the active list (every instance in ids, all alive) for rows-per-
// tile ty, resets the pass counters and empties the request ring.
eik_status upload_list(BatchExec *e, const std::vector<int> &ids, int ty) {
  std::vector<int> act(ids), pre(ids.size() + 1, 0), alive(e->count, 0);
  for (size_t a = 0; a < ids.size(); ++a) {
    pre[a + 1] = pre[a] + tiles_of(e->h_bi[ids[a]], ty);
    alive[ids[a]] = 1;
  }
  if (pre.back() > e->part_cap) {
    e->msg = "packed batch: tile list exceeds the partials buffer";
    return EIK_ERR_ARG;
  }
  BatchCtl c{};
  c.m = (int)ids.size();
  c.ntiles = pre.back();
  *e->h_bc = c;
  e->ring->tail = 0;
  e->pushed = 0;
  if (!act.empty())
    BCK(cudaMemcpyAsync(e->act, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice,
                        e->stream));
  BCK(cudaMemcpyAsync(e->pre, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice,
                      e->stream));
  BCK(cudaMemcpyAsync(e->alive, alive.data(), sizeof(int) * e->count, cudaMemcpyHostToDevice,
                      e->stream));
  BCK(cudaMemcpyAsync(e->bc, e->h_bc, sizeof(BatchCtl), cudaMemcpyHostToDevice, e->stream));
  BCK(cudaMemsetAsync(e->cnt, 0, sizeof(unsigned) * e->count, e->stream));
  // the host-side list and control block must outlive the copies
  BCK(cudaStreamSynchronize(e->stream));
  return EIK_OK;
}

eik_status upload_bi(BatchExec *e) {
  if (!e->bi_dirty) return EIK_OK;
  BCK(cudaMemcpyAsync(e->bi, e->h_bi.data(), sizeof(BInst) * e->count, cudaMemcpyHostToDevice,
                      e->stream));
  BCK(cudaStreamSynchronize(e->stream));
  e->bi_dirty = false;
  return EIK_OK;
}

eik_status set_plan(BatchExec *e, int variant, int ty) {
  const char *why = "";
  if (!cg32_batch_plan(&e->plan, e->bufs, e->num_sms, variant, ty, &why)) {
    e->msg = std::string("packed batch: ") + why;
    return EIK_ERR_CUDA;
  }
  if (e->graph) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
  }
  return EIK_OK;
}

// Times every candidate tile shape on a synthetic state of this batch's
// geometry (all instances active, none converging) and keeps the fastest.
eik_status tune(BatchExec *e) {
  std::vector<int> vars, tys;
  for (int v = 1; v <= 4; ++v)
    if (e->variant_req == 0 || e->variant_req == v) vars.push_back(v);
  if (e->ty_req > 0)
    tys.push_back(e->ty_req);
  else
    tys.assign(std::begin(kTuneTy), std::end(kTuneTy));
  // kx = 0 for the timing (each instance writes its own at setup)
  for (int i = 0; i < e->count; ++i)
    if (e->h_bi[i].kx)
      BCK(cudaMemsetAsync(const_cast<int *>(e->h_bi[i].kx), 0, sizeof(int) * e->cells[i],
                          e->stream));
  const int64_t total = (int64_t)e->P * e->H;
  k_tune_fill<<<e->num_sms * 8, 256, 0, e->stream>>>(total, e->P, e->row_inst, e->bi, e->arr[0],
                                                      e->arr[4]);
  BCK(cudaGetLastError());
  std::vector<MixCtl> ctl(e->count);
  for (auto &c : ctl) {
    c = MixCtl{};
    c.gam_m = 1.0;
    c.mode = 0;
    c.thresh = -1.f;
    c.max_iter = INT_MAX;
    c.first = 1;
  }
  std::vector<int> all(e->count);
  for (int i = 0; i < e->count; ++i) all[i] = i;
  cudaEvent_t ev0, ev1;
  BCK(cudaEventCreate(&ev0));
  BCK(cudaEventCreate(&ev1));
  double best = INFINITY;
  int bv = 1, bt = tys[0];
  for (int v : vars)
    for (int ty : tys) {
      if (set_plan(e, v, ty) != EIK_OK) {
        cudaGetLastError();
        continue;
      }
      BCK(cudaMemcpyAsync(e->st, ctl.data(), sizeof(MixCtl) * e->count, cudaMemcpyHostToDevice,
                          e->stream));
      eik_status ls = upload_list(e, all, ty);
      if (ls != EIK_OK) return ls;
      for (int k = 0; k <= kTuneWarm; ++k) cg32_batch_pass(e->plan, e->bufs, k & 1, e->stream);
      BCK(cudaEventRecord(ev0, e->stream));
      for (int k = 0; k < kTuneTimed; ++k)
        cg32_batch_pass(e->plan, e->bufs, (kTuneWarm + 1 + k) & 1, e->stream);
      BCK(cudaEventRecord(ev1, e->stream));
      BCK(cudaGetLastError());
      BCK(cudaStreamSynchronize(e->stream));
      e->passes += 1 + kTuneWarm + kTuneTimed;
      BCK(cudaMemcpy(e->h_bc, e->bc, sizeof(BatchCtl), cudaMemcpyDeviceToHost));
      if (e->h_bc->fault) {
        e->msg = "packed batch: a device-side wait for a tile copy timed out while tuning";
        return EIK_ERR_TIMEOUT;
      }
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, ev0, ev1));
      const double us = 1e3 * ms / kTuneTimed;
      if (getenv("EIK_TRACE_BATCH"))
        fprintf(stderr, "[batch] tune variant %d ty %d: %.1f us per pass (%d instances active)\n",
                v, ty, us, e->h_bc->m);
      if (us < best) {
        best = us;
        bv = v;
        bt = ty;
      }
    }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (!std::isfinite(best)) {
    e->msg = "packed batch: no tile shape could be configured";
    return EIK_ERR_CUDA;
  }
  eik_status ps = set_plan(e, bv, bt);
  if (ps != EIK_OK) return ps;
  const std::string path = cache_path();
  if (!path.empty()) {
    auto m = cache_read(path);
    m[tune_key(e)] = TuneEntry{bv, bt, best};
    cache_write(path, m);
  }
  return EIK_OK;
}

eik_status ensure_plan(BatchExec *e) {
  if (e->planned) return EIK_OK;
  eik_status s = upload_bi(e);
  if (s != EIK_OK) return s;
  if (e->variant_req > 0 && e->ty_req > 0) {
    s = set_plan(e, e->variant_req, e->ty_req);
    e->how = 0;
  } else {
    const std::string path = cache_path();
    bool hit = false;
    if (!path.empty()) {
      const auto m = cache_read(path);
      const auto it = m.find(tune_key(e));
      if (it != m.end() && (e->variant_req == 0 || e->variant_req == it->second.variant) &&
          (e->ty_req == 0 || e->ty_req == it->second.ty)) {
        s = set_plan(e, it->second.variant, it->second.ty);
        hit = s == EIK_OK;
        e->how = 2;
      }
    }
    if (!hit) {
      s = tune(e);
      e->how = 1;
    }
  }
  if (s == EIK_OK) e->planned = true;
  return s;
}

eik_status build_graph(BatchExec *e) {
  if (e->graph) return EIK_OK;
  cudaGraph_t g;
  BCK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < kGraphPasses; ++k) cg32_batch_pass(e->plan, e->bufs, k & 1, e->stream);
  BCK(cudaStreamEndCapture(e->stream, &g));
  const cudaError_t ie = cudaGraphInstantiate(&e->graph, g, 0);
  cudaGraphDestroy(g);
  BCK(ie);
  return EIK_OK;
}

// Executor: graphs of passes while an instance iterates or a request waits;
// idle (on the condition variable) otherwise; ends when no program is left.
eik_status exec_run(BatchExec *e) {
  BCK(cudaSetDevice(e->device));
  bool active = false;
  int admitted = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(e->mu);
      for (;;) {
        if (active || e->pushed > admitted) break;
        if (e->live == 0) return EIK_OK;
        e->cv.wait_for(lk, std::chrono::milliseconds(2));
      }
    }
    BCK(cudaEventRecord(e->ev[0], e->stream));
    BCK(cudaGraphLaunch(e->graph, e->stream));
    BCK(cudaEventRecord(e->ev[1], e->stream));
    BCK(cudaMemcpyAsync(e->h_bc, e->bc, sizeof(BatchCtl), cudaMemcpyDeviceToHost, e->stream));
    BCK(cudaStreamSynchronize(e->stream));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, e->ev[0], e->ev[1]));
    e->pass_ms += ms;
    if (e->h_bc->fault) {
      e->msg = "a device-side wait for a tile copy timed out";
      return EIK_ERR_TIMEOUT;
    }
    active = e->h_bc->m > 0;
    admitted = e->h_bc->req_head;
  }
}

void exec_main(BatchExec *e) {
  const eik_status s = exec_run(e);
  if (s != EIK_OK) {
    e->exec_status = s;
    e->abort.store(1, std::memory_order_release);
  }
}

}  // namespace

eik_status batch_exec_create(BatchExec **out, int count, const int *nx, const int *ny,
                             int boundary, int num_sms, int variant, int ty) {
  *out = nullptr;
  if (count < 1 || variant < 0 || variant > 4 || ty < 0 || ty > 1024) return EIK_ERR_ARG;
  BatchExec *e = new BatchExec();
  e->count = count;
  e->num_sms = num_sms;
  e->boundary = boundary;
  e->variant_req = variant;
  e->ty_req = ty;
  e->h_bi.resize(count);
  e->cells.assign(count, 0);
  e->seq.assign(count, 0);
  cudaGetDevice(&e->device);
  int maxw = 4;
  int64_t rows = 2;
  int64_t cap = 0;
  const int tymin = (ty > 0) ? ty : kTuneTy[0];
  for (int i = 0; i < count; ++i) {
    BInst &b = e->h_bi[i];
    b = BInst{};
    b.nx = nx[i];
    b.ny = ny[i];
    b.wx = (nx[i] + 3) / 4 * 4;
    b.row0 = (int)rows;
    b.tiles_x = (nx[i] + 127) / 128;
    b.boundary = boundary;
    maxw = std::max(maxw, b.wx);
    rows += (int64_t)ny[i] + 2;   // two zero rows after every instance
    cap += tiles_of(b, tymin);
    e->nodes += (int64_t)nx[i] * ny[i];
  }
  if (rows > INT_MAX / 2 || cap > INT_MAX / 8) {
    delete e;
    return EIK_ERR_ARG;
  }
  e->P = maxw;
  e->H = (int)rows;
  e->part_cap = (int)cap;
  const size_t ne = (size_t)e->P * e->H;
  bool ok = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 7 && ok; ++k) {
    ok = cudaMalloc((void **)&e->arr[k], sizeof(float) * ne) == cudaSuccess;
    ok = ok && cudaMemsetAsync(e->arr[k], 0, sizeof(float) * ne, e->stream) == cudaSuccess;
  }
  ok = ok && cudaMalloc((void **)&e->bi, sizeof(BInst) * count) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->st, sizeof(MixCtl) * count) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->act, sizeof(int) * count) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->pre, sizeof(int) * (count + 1)) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->cnt, sizeof(unsigned) * count) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->row_inst, sizeof(int) * e->H) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->bc, sizeof(BatchCtl)) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->part, sizeof(double) * 6 * (size_t)cap) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&e->alive, sizeof(int) * count) == cudaSuccess;
  ok = ok && cudaEventCreate(&e->ev[0]) == cudaSuccess && cudaEventCreate(&e->ev[1]) == cudaSuccess;
  ok = ok && cudaMallocHost((void **)&e->h_bc, sizeof(BatchCtl)) == cudaSuccess;
  ok = ok && cudaHostAlloc((void **)&e->ring, sizeof(BatchRing) + sizeof(int) * count,
                           cudaHostAllocMapped) == cudaSuccess;
  ok = ok && cudaHostAlloc((void **)&e->done, sizeof(BatchDone) * count, cudaHostAllocMapped) ==
                 cudaSuccess;
  ok = ok && cudaHostGetDevicePointer((void **)&e->d_ring, e->ring, 0) == cudaSuccess;
  ok = ok && cudaHostGetDevicePointer((void **)&e->d_done, e->done, 0) == cudaSuccess;
  if (ok) {
    memset((void *)e->ring, 0, sizeof(BatchRing) + sizeof(int) * count);
    memset((void *)e->done, 0, sizeof(BatchDone) * count);
  }
  if (ok) {
    std::vector<int> ri(e->H, -1);
    for (int i = 0; i < count; ++i)
      for (int y = 0; y < ny[i]; ++y) ri[e->h_bi[i].row0 + y] = i;
    ok = cudaMemsetAsync(e->st, 0, sizeof(MixCtl) * count, e->stream) == cudaSuccess &&
         cudaMemsetAsync(e->bc, 0, sizeof(BatchCtl), e->stream) == cudaSuccess &&
         cudaMemsetAsync(e->cnt, 0, sizeof(unsigned) * count, e->stream) == cudaSuccess &&
         cudaMemsetAsync(e->alive, 0, sizeof(int) * count, e->stream) == cudaSuccess &&
         cudaMemcpyAsync(e->row_inst, ri.data(), sizeof(int) * e->H, cudaMemcpyHostToDevice,
                         e->stream) == cudaSuccess &&
         cudaStreamSynchronize(e->stream) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    batch_exec_destroy(e);
    return EIK_ERR_OOM;
  }
  Cg32BatchBuffers &b = e->bufs;
  b.r[0] = e->arr[0];
  b.r[1] = e->arr[1];
  b.p[0] = e->arr[2];
  b.p[1] = e->arr[3];
  b.s32 = e->arr[4];
  b.d = e->arr[5];
  b.xref = e->arr[6];
  b.P = e->P;
  b.H = e->H;
  b.bi = e->bi;
  b.st = e->st;
  b.act = e->act;
  b.pre = e->pre;
  b.cnt = e->cnt;
  b.bc = e->bc;
  b.part = e->part;
  b.part_cap = e->part_cap;
  b.alive = e->alive;
  b.ring = e->d_ring;
  b.ring_cap = count;
  b.done = e->d_done;
  *out = e;
  return EIK_OK;
}

void batch_exec_destroy(BatchExec *e) {
  if (!e) return;
  if (e->exec.joinable()) {
    {
      std::lock_guard<std::mutex> lk(e->mu);
      e->live = 0;
    }
    e->cv.notify_all();
    e->exec.join();
  }
  if (e->stream) cudaStreamSynchronize(e->stream);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  for (float *a : e->arr)
    if (a) cudaFree(a);
  void *ptrs[] = {e->bi, e->st, e->act, e->pre, e->cnt, e->row_inst, e->bc, e->part, e->alive};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t ev : e->ev)
    if (ev) cudaEventDestroy(ev);
  if (e->h_bc) cudaFreeHost(e->h_bc);
  if (e->ring) cudaFreeHost((void *)e->ring);
  if (e->done) cudaFreeHost(e->done);
  if (e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

BatchMember batch_exec_member(BatchExec *e, int i) {
  const int64_t off = (int64_t)e->h_bi[i].row0 * e->P;
  return BatchMember{e->arr[0] + off, e->arr[2] + off, e->arr[4] + off, e->arr[5] + off,
                     e->arr[6] + off, e->P,           e->st + i};
}

void batch_exec_set_cells(BatchExec *e, int i, const CellGrid &cg, const int *kx) {
  e->h_bi[i].cg = cg;
  e->h_bi[i].kx = kx;
  e->cells[i] = cg.ncell;
  e->bi_dirty = true;
}

eik_status batch_exec_begin(BatchExec *e, int live) {
  if (e->exec.joinable()) {
    e->msg = "packed batch: a solve is already running";
    return EIK_ERR_STATE;
  }
  eik_status s = ensure_plan(e);
  if (s != EIK_OK) return s;
  s = upload_list(e, std::vector<int>(), e->plan.ty);   // empty list, empty ring
  if (s != EIK_OK) return s;
  s = build_graph(e);
  if (s != EIK_OK) return s;
  e->live = live;
  e->abort.store(0);
  e->exec_status = EIK_OK;
  e->exec = std::thread(exec_main, e);
  return EIK_OK;
}

int batch_exec_ticket(BatchExec *e, int i) {
  std::lock_guard<std::mutex> lk(e->mu);
  return ++e->seq[i];
}

eik_status batch_exec_inner(BatchExec *e, int i, int seq, MixCtl *out) {
  {
    std::lock_guard<std::mutex> lk(e->mu);
    const int t = e->pushed;
    e->ring->ids[t % e->count] = i;
    std::atomic_thread_fence(std::memory_order_release);
    e->ring->tail = t + 1;
    e->pushed = t + 1;
  }
  e->cv.notify_all();
  volatile BatchDone *d = e->done + i;
  for (int spin = 0; d->done_seq != seq; ++spin) {
    // the executor wrote its status and message before raising abort, and
    // writes neither afterwards
    if (e->abort.load(std::memory_order_acquire))
      return e->exec_status != EIK_OK ? e->exec_status : EIK_ERR_CUDA;
    if (spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  out->iter = d->iter;
  out->status = d->status;
  out->stalled = d->stalled;
  out->alpha = d->alpha;
  out->beta = d->beta;
  out->F = d->F;
  out->done = 1;
  return EIK_OK;
}

void batch_exec_leave(BatchExec *e, int i) {
  (void)i;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    --e->live;
  }
  e->cv.notify_all();
}

eik_status batch_exec_end(BatchExec *e) {
  if (e->exec.joinable()) e->exec.join();
  e->passes += e->h_bc->passes;
  e->work += e->h_bc->work;
  return e->exec_status;
}

void batch_exec_plan(const BatchExec *e, int *variant, int *ty, int *how) {
  *variant = e->planned ? e->plan.variant : 0;
  *ty = e->planned ? e->plan.ty : 0;
  *how = e->how;
}

int64_t batch_exec_passes(const BatchExec *e) { return e->passes; }

void batch_exec_work(const BatchExec *e, int64_t *node_passes, double *ms) {
  *node_passes = e->work;
  *ms = e->pass_ms;
}

std::string batch_exec_error(const BatchExec *e) {
  return e->msg.empty() ? std::string("packed batch executor stopped") : e->msg;
}

}  // namespace eik
