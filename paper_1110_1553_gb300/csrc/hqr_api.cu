// C ABI of the library (include/hqr.h): argument checks, workspace and task
// graph management, and the launches of the device engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/hqr.h"
#include "engine.cuh"
#include "hqr_internal.h"

using namespace hqr;

namespace {

thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;
int64_t g_timeout_ns = 20000000000ll;

bool cuda_ok(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  (void)cudaGetLastError();  // a non-sticky error must not be reported again by a later launch check
  return false;
}
#define CK(call)                                      \
  do {                                                \
    if (!cuda_ok((call), #call)) return HQR_ERR_CUDA; \
  } while (0)

// A task graph resident on the device, with pristine copies of the
// in-degrees, the ready slots and the control words for every new run.
struct DevGraph {
  Task *tasks = nullptr;
  int *succ = nullptr;
  int *indeg0 = nullptr, *indeg = nullptr;
  int *slots0 = nullptr, *slots = nullptr;
  Ctl *ctl0 = nullptr, *ctl = nullptr;
  int ntasks = 0;
  int64_t nedges = 0;
  void release() {
    cudaFree(tasks);
    cudaFree(succ);
    cudaFree(indeg0);
    cudaFree(indeg);
    cudaFree(slots0);
    cudaFree(slots);
    cudaFree(ctl0);
    cudaFree(ctl);
    *this = DevGraph();
  }
};

// Setup copies and fills go through the legacy default stream, while the
// kernels may run on any stream, non-blocking ones (and the server's own)
// included, which that stream does not order: setup waits for it before
// anything is launched.
int setup_done() {
  CK(cudaStreamSynchronize(cudaStreamLegacy));
  return HQR_SUCCESS;
}

int upload_graph(const Graph &g, DevGraph &d) {
  const int nt = (int)g.tasks.size();
  d.ntasks = nt;
  d.nedges = g.nedges;
  std::vector<int> slots(slot_count(nt), 0);
  std::vector<Ctl> ctlv(1);
  Ctl &ctl = ctlv[0];
  init_ready(g.tasks.data(), g.indeg.data(), nt, slots.data(), ctl);
  const size_t ns = std::max<size_t>(g.succ.size(), 1);
  CK(cudaMalloc(&d.tasks, sizeof(Task) * nt));
  CK(cudaMalloc(&d.succ, sizeof(int) * ns));
  CK(cudaMalloc(&d.indeg0, sizeof(int) * nt));
  CK(cudaMalloc(&d.indeg, sizeof(int) * nt));
  CK(cudaMalloc(&d.slots0, sizeof(int) * slots.size()));
  CK(cudaMalloc(&d.slots, sizeof(int) * slots.size()));
  CK(cudaMalloc(&d.ctl0, sizeof(Ctl)));
  CK(cudaMalloc(&d.ctl, sizeof(Ctl)));
  CK(cudaMemcpy(d.tasks, g.tasks.data(), sizeof(Task) * nt, cudaMemcpyHostToDevice));
  if (!g.succ.empty())
    CK(cudaMemcpy(d.succ, g.succ.data(), sizeof(int) * g.succ.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.indeg0, g.indeg.data(), sizeof(int) * nt, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.slots0, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d.ctl0, &ctl, sizeof(Ctl), cudaMemcpyHostToDevice));
  return setup_done();
}

// Tile-major packing of a column-major matrix, zero padded to whole tiles.
template <typename Real>
__global__ void pack_tiles(const Real *__restrict__ A, long long lda, int M, int N, Real *__restrict__ ws, int m,
                           int nb, long long total) {
  const long long nb2 = (long long)nb * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long tile = e / nb2;
    const int w = (int)(e - tile * nb2);
    const int cc = w / nb, rr = w - cc * nb;
    const int ti = (int)(tile % m), tj = (int)(tile / m);
    const int row = ti * nb + rr, col = tj * nb + cc;
    ws[e] = (row < M && col < N) ? A[(long long)col * lda + row] : Real(0);
  }
}

// Inverse of pack_tiles for the leading rows x cols of the padded matrix;
// `upper_only` keeps rows <= col and zeroes the rest (R).
template <typename Real>
__global__ void unpack_tiles(const Real *__restrict__ ws, int m, int nb, Real *__restrict__ out, long long ld,
                             int rows, int cols, int upper_only) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(e / rows), row = (int)(e - (long long)col * rows);
    const int ti = row / nb, tj = col / nb;
    Real v = ws[((size_t)tj * m + ti) * nb * nb + (size_t)(col - tj * nb) * nb + (row - ti * nb)];
    if (upper_only && row > col) v = 0;
    out[(long long)col * ld + row] = v;
  }
}

// Right-hand side (M x nrhs) into blocks of nb rows x wa columns: block
// (r, s) at ((s*m + r)*nb*wa), column-major inside.
template <typename Real>
__global__ void pack_rhs(const Real *__restrict__ B, long long ldb, int M, int nrhs, Real *__restrict__ Bw, int m,
                         int nb, int wa, long long total) {
  const long long bs = (long long)nb * wa;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / bs;
    const int w = (int)(e - blk * bs);
    const int cc = w / nb, rr = w - cc * nb;
    const int r = (int)(blk % m), s = (int)(blk / m);
    const int row = r * nb + rr, col = s * wa + cc;
    Bw[e] = (row < M && col < nrhs) ? B[(long long)col * ldb + row] : Real(0);
  }
}

template <typename Real>
__global__ void unpack_rhs(const Real *__restrict__ Bw, Real *__restrict__ B, long long ldb, int M, int nrhs, int m,
                           int nb, int wa) {
  const long long total = (long long)M * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(e / M), row = (int)(e - (long long)col * M);
    const int r = row / nb, rr = row - r * nb, s = col / wa, cc = col - s * wa;
    B[(long long)col * ldb + row] = Bw[((size_t)s * m + r) * nb * wa + (size_t)cc * nb + rr];
  }
}

// Back substitution with the diagonal tile i (nbi x nbi leading part), one
// CTA per right-hand side; x holds c on entry.
template <typename Real>
__global__ void trsv_diag(const Real *__restrict__ ws, int m, int nb, int i, int nbi, Real *X, long long ldx,
                          int *singular) {
  __shared__ Real xs[256];
  Real *x = X + (long long)blockIdx.x * ldx + (long long)i * nb;
  const Real *Rt = ws + ((size_t)i * m + i) * nb * nb;
  for (int r = threadIdx.x; r < nbi; r += blockDim.x) xs[r] = x[r];
  __syncthreads();
  for (int r = nbi - 1; r >= 0; --r) {
    if (threadIdx.x == 0) {
      const Real d = Rt[(size_t)r * nb + r];
      if (d == Real(0)) {
        atomicExch(singular, 1);
        xs[r] = 0;
      } else {
        xs[r] = xs[r] / d;
      }
    }
    __syncthreads();
    const Real xr = xs[r];
    for (int l = threadIdx.x; l < r; l += blockDim.x) xs[l] = fma(-Rt[(size_t)r * nb + l], xr, xs[l]);
    __syncthreads();
  }
  for (int r = threadIdx.x; r < nbi; r += blockDim.x) x[r] = xs[r];
}

// c[0 : i*nb) -= R[0 : i*nb, columns of tile i] x_i.
template <typename Real>
__global__ void trsv_update(const Real *__restrict__ ws, int m, int nb, int i, int nbi, Real *X, long long ldx) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= i * nb) return;
  const int ti = row / nb, rr = row - ti * nb;
  const Real *Rt = ws + ((size_t)i * m + ti) * nb * nb;
  const Real *x = X + (long long)blockIdx.y * ldx + (long long)i * nb;
  Real s = 0;
  for (int c = 0; c < nbi; ++c) s = fma(Rt[(size_t)c * nb + rr], x[c], s);
  X[(long long)blockIdx.y * ldx + row] -= s;
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>(4096, (n + 255) / 256)); }

size_t elem_size(int prec) { return prec == HQR_FP64 ? sizeof(double) : sizeof(float); }

// The persistent scheduler instantiation for a storage precision (and the
// tensor-core variant for graphs that hold tensor-core problems).
const void *sched_kernel(int prec, bool tc) {
  if (prec == HQR_FP64) return (const void *)hqr_sched<double, false>;
  return tc ? (const void *)hqr_sched<float, true> : (const void *)hqr_sched<float, false>;
}

size_t smem_for(int prec, const Problem &P) {
  if (P.tc) return engine_smem_bytes_tc();
  const int wmax = std::max(P.w, P.wb);
  return prec == HQR_FP64 ? engine_smem_bytes<double>(P.nb, P.ib, wmax, P.wt, P.vc)
                          : engine_smem_bytes<float>(P.nb, P.ib, wmax, P.wt, P.vc);
}

// CTAs for a launch: every SM filled to the occupancy the kernel allows.
int ctas_for(int prec, bool tc, size_t smem, int ntasks, int *grid) {
  static size_t attr[3] = {0, 0, 0};
  const void *k = sched_kernel(prec, tc);
  const int slot = prec == HQR_FP64 ? 0 : (tc ? 2 : 1);
  if (attr[slot] < smem) {
    CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[slot] = smem;
  }
  int dev = 0, sms = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
  if (per_sm < 1) {
    g_last_error = "scheduler kernel does not fit on an SM";
    return HQR_ERR_CUDA;
  }
  *grid = std::max(1, std::min(sms * per_sm, ntasks));
  return HQR_SUCCESS;
}

int launch_sched(int prec, const EngineParams &p, size_t smem, cudaStream_t s, int max_ctas = 0) {
  if (p.tc && smem < engine_smem_bytes_tc()) {  // the tensor-core tasks lay out that much shared memory
    g_last_error = "tensor-core launch with too little shared memory";
    return HQR_ERR_INTERNAL;
  }
  int grid = 0;
  int st = ctas_for(prec, p.tc != 0, smem, p.ntasks, &grid);
  if (st) return st;
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  if (prec == HQR_FP64)
    hqr_sched<double, false><<<grid, NT, smem, s>>>(p);
  else if (p.tc)
    hqr_sched<float, true><<<grid, NT, smem, s>>>(p);
  else
    hqr_sched<float, false><<<grid, NT, smem, s>>>(p);
  CK(cudaGetLastError());
  g_launches += 1;
  return HQR_SUCCESS;
}

// Explicit slab widths (0 = built-in choice), set by hqr_set_slab_widths.
int g_w_override = 0, g_wt_override = 0, g_vc_override = 0;
// Priority policy of task graphs (hqr_set_priority_policy).
int g_priority_policy = 1;
// CUDA-core panels of tiles with nb >= this are split into block tasks (hqr_set_panel_split; 0: never).
int g_split_min_nb = 64;
// Plans with tensor-core and CUDA-core problems launch them side by side (hqr_set_split_launch).
int g_split_launch = 1;

// Block size of a split panel for a problem, or 0 to keep whole panel tasks. The tensor-core
// kernels keep whole panels (one block per tile). FP32 panels on CUDA cores are cheap next to
// their updates: they are split only where a block spans whole update slabs (measured: splitting
// blocks narrower than the 64-column FP32 slabs cost 1024 uneven problems 5 %); FP64 panels are
// split at any slab width (512^2 FP64 QR + Q: -25 % latency).
int split_ib_for(int prec, const Problem &P) {
  if (P.tc || g_split_min_nb <= 0 || P.nb < g_split_min_nb) return 0;
  if (P.w <= 0 || P.nb / P.ib < 2) return 0;
  if (prec != HQR_FP64 && P.ib % P.w != 0) return 0;
  return P.ib;
}

// Tuning of the column-slab widths for a tile size and precision. FP64 work
// is bound by the FP64 pipe, so narrow slabs (more parallel tasks) cost
// nothing; FP32 tasks are bound by their barriers and staging, so they take
// wider slabs (more arithmetic per barrier) within the shared memory of two
// CTAs per SM.
bool prec_ok(int prec) { return prec == HQR_FP64 || prec == HQR_FP32 || prec == HQR_FP32_BF16X3; }

// Tiles of this size on the tensor-core kernels (with one full T per tile).
bool use_tc(int prec, int nb) { return prec == HQR_FP32_BF16X3 && nb == tc::NB; }

// Inner block of the T factors: the tensor-core path keeps one full T.
int eff_ib(int prec, int nb, int ib) { return use_tc(prec, nb) ? nb : ib; }

// Elements of one T record (the T factor; tensor-core tiles add the split
// operand images of their updates).
size_t t_record(int prec, int nb, int ib, bool t32 = true) {
  if (!use_tc(prec, nb)) return (size_t)ib * nb;
  return t32 ? (size_t)tc::T_RECORD : (size_t)tc::T_RECORD_IMG;
}

// Least-squares problems (plans, server) apply only Q^T: their tensor-core T
// records leave out the FP32 T.
void drop_t32(int prec, Problem &P) {
  P.t32 = 0;
  P.tstr = (int)t_record(prec, P.nb, P.ib, false);
}

void choose_widths(int prec, int nb, int ib, Problem &P) {
  P.wb = std::min(16, nb);
  P.tc = use_tc(prec, nb) ? 1 : 0;
  P.t32 = 1;
  P.tstr = (int)t_record(prec, nb, ib);
  if (P.tc) {
    P.w = tc::WMAX;
    P.wt = 32;
    P.vc = 16;
    return;
  }
  if (prec == HQR_FP64) {
    P.w = std::min(16, nb);
    P.wt = nb > 128 ? 8 : std::min(16, nb);
    P.vc = nb > 128 ? std::min(ib, 8) : std::min(ib, 16);
  } else {
    P.w = nb >= 256 ? 32 : std::min(64, nb);
    P.wt = nb >= 256 ? 16 : std::min(32, nb);
    P.vc = std::min(ib, 16);
  }
  if (g_w_override > 0) P.w = std::min(g_w_override, nb);
  if (g_wt_override > 0) P.wt = std::min(g_wt_override, nb);
  if (g_vc_override > 0 && ib % g_vc_override == 0) P.vc = std::min(g_vc_override, ib);
}

bool valid_tile_sizes(int prec, int nb, int ib) {
  if (use_tc(prec, nb)) return ib == nb;
  if (nb < 8 || nb > 256 || nb % 8) return false;
  const int align = prec == HQR_FP64 ? 2 : 4;  // rows per 16 bytes
  if (ib < align || ib % align || nb % ib || (ib > 16 && ib != 32)) return false;
  return true;
}

}  // namespace

struct hqr_factors {
  int M = 0, N = 0, Mp = 0, Np = 0, m = 0, n = 0, nb = 0, ib = 0, prec = 0;
  std::vector<hqr_elim_t> list;
  std::vector<PanelOp> ops;
  Problem prob{};        // host copy of the device descriptor
  Problem *dprob = nullptr;
  void *dA = nullptr, *dT = nullptr, *dBw = nullptr;
  size_t bw_cap = 0;
  DevGraph fg;
  std::map<std::pair<int, int>, DevGraph> ag;  // (trans, nslab) -> apply graph
  Ctl *last_ctl = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  // start / end events of the last kRing task-kernel runs (hqr_kernel_times)
  static constexpr int kRing = 64;
  std::vector<cudaEvent_t> ring;
  int64_t ring_runs = 0, ring_read = 0;
  unsigned long long *dtrace = nullptr;
  size_t trace_cap = 0;
  int64_t debug_task = -1;
  int debug_base = -1;
};

namespace {

int run_graph(hqr_factors *F, DevGraph &g, cudaStream_t s) {
  EngineParams p{};
  p.tc = F->prob.tc;
  p.probs = F->dprob;
  p.tasks = g.tasks;
  p.ntasks = g.ntasks;
  p.succ = g.succ;
  p.indeg = g.indeg;
  p.slots = g.slots;
  p.ctl = g.ctl;
  p.timeout_ns = g_timeout_ns;
  p.trace = (F->dtrace && F->trace_cap >= (size_t)g.ntasks) ? F->dtrace : nullptr;
  const size_t smem = smem_for(F->prec, F->prob);
  CK(cudaMemcpyAsync(g.indeg, g.indeg0, sizeof(int) * g.ntasks, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(g.slots, g.slots0, sizeof(int) * slot_count(g.ntasks), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(g.ctl, g.ctl0, sizeof(Ctl), cudaMemcpyDeviceToDevice, s));
  if (!F->ev0) {
    CK(cudaEventCreate(&F->ev0));
    CK(cudaEventCreate(&F->ev1));
  }
  if (F->ring.empty()) {
    F->ring.assign(2 * hqr_factors::kRing, nullptr);
    for (cudaEvent_t &e : F->ring) CK(cudaEventCreate(&e));
  }
  const int slot = (int)(F->ring_runs % hqr_factors::kRing);
  CK(cudaEventRecord(F->ev0, s));
  CK(cudaEventRecord(F->ring[2 * slot], s));
  int st = launch_sched(F->prec, p, smem, s);
  if (st) return st;
  CK(cudaEventRecord(F->ev1, s));
  CK(cudaEventRecord(F->ring[2 * slot + 1], s));
  F->ring_runs += 1;
  F->timed = true;
  F->last_ctl = g.ctl;
  return HQR_SUCCESS;
}

int read_status(hqr_factors *F, cudaStream_t s) {
  CK(cudaStreamSynchronize(s));
  if (!F->last_ctl) return HQR_SUCCESS;
  CtlLine c;
  CK(cudaMemcpy(&c, &F->last_ctl->status, sizeof(CtlLine), cudaMemcpyDeviceToHost));
  if (c.v != 0) return (int)c.v;
  return HQR_SUCCESS;
}

int pack_a(hqr_factors *F, const void *dA, int lda, cudaStream_t s) {
  const long long total = (long long)F->Mp * F->Np;
  if (F->prec == HQR_FP64)
    pack_tiles<double><<<grid_for(total), 256, 0, s>>>((const double *)dA, lda, F->M, F->N, (double *)F->dA,
                                                       F->m, F->nb, total);
  else
    pack_tiles<float><<<grid_for(total), 256, 0, s>>>((const float *)dA, lda, F->M, F->N, (float *)F->dA, F->m,
                                                      F->nb, total);
  CK(cudaGetLastError());
  g_launches += 1;
  return HQR_SUCCESS;
}

int push_problem(hqr_factors *F) {
  F->prob.A = F->dA;
  F->prob.T = F->dT;
  F->prob.B = F->dBw;
  if (!F->dprob) CK(cudaMalloc(&F->dprob, sizeof(Problem)));
  CK(cudaMemcpy(F->dprob, &F->prob, sizeof(Problem), cudaMemcpyHostToDevice));
  return setup_done();
}

}  // namespace

extern "C" {

void hqr_set_timeout_ms(int64_t ms) { g_timeout_ns = (ms > 0 ? ms : 1) * 1000000ll; }

int hqr_set_priority_policy(int policy) {
  if (policy != 0 && policy != 1) return -1;
  g_priority_policy = policy;
  return HQR_SUCCESS;
}

int hqr_set_split_launch(int on) {
  if (on < 0 || on > 1) return -1;
  g_split_launch = on;
  return HQR_SUCCESS;
}

int hqr_set_panel_split(int min_nb) {
  if (min_nb < 0) return -1;
  g_split_min_nb = min_nb;
  return HQR_SUCCESS;
}

int hqr_set_slab_widths(int w, int wt, int vc) {
  if (w < 0 || w % 2) return -1;
  if (wt < 0 || wt % 2) return -2;
  if (vc < 0 || (vc && vc % 2)) return -3;
  g_w_override = w;
  g_wt_override = wt;
  g_vc_override = vc;
  return HQR_SUCCESS;
}

const char *hqr_last_error(void) { return g_last_error.c_str(); }

int64_t hqr_last_launches(void) { return g_launches; }

const char *hqr_strerror(int status) {
  switch (status) {
    case HQR_SUCCESS: return "success";
    case HQR_ERR_CUDA: return "CUDA error";
    case HQR_ERR_TIMEOUT: return "device wait timed out";
    case HQR_ERR_NOMEM: return "out of memory";
    case HQR_ERR_CAPACITY: return "output array too small";
    case HQR_ERR_INVALID_LIST: return "invalid elimination list";
    case HQR_ERR_SINGULAR: return "R has an exact zero on its diagonal";
    case HQR_ERR_INTERNAL: return "internal error";
    case HQR_ERR_TOO_LARGE: return "problem exceeds the limits of the allocation-free entry point";
    case HQR_ERR_BUSY: return "no room for the request right now";
    case HQR_ERR_BUDGET: return "request exceeds the server's budget";
    case HQR_ERR_NOCONV: return "refinement did not reach the tolerance";
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

}  // extern "C"
namespace {
int na_task_graph(int m, int n, int nb, int ib, const hqr_elim_t *list, size_t count, int32_t *tasks,
                  int64_t task_cap, int64_t *succ_ptr, int32_t *succ, int64_t succ_cap, int64_t *ntasks,
                  int64_t *nedges);
}  // namespace
extern "C" {

int hqr_task_graph(int m, int n, int nb, int ib, int prec, const hqr_elim_t *list, size_t count, int kind,
                   int param, int32_t *tasks, int64_t task_cap, int64_t *succ_ptr, int32_t *succ, int64_t succ_cap,
                   int64_t *ntasks, int64_t *nedges) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (!prec_ok(prec)) return -5;
  if (nb < 8 || nb > 256 || nb % 8 || (prec == HQR_FP32_BF16X3 && nb != tc::NB)) return -3;
  ib = eff_ib(prec, nb, ib);
  if (!valid_tile_sizes(prec, nb, ib)) return -4;
  if (!list && count) return -6;
  if (kind < 0 || kind > 6) return -8;
  if (kind == 6 && prec != HQR_FP64) return -5;
  if (param < 0 || ((kind == 1 || kind == 2) && param < 1)) return -9;
  if (!ntasks || !nedges) return -16;
  if (hqr_validate_list(m, n, list, count) != HQR_SUCCESS) return HQR_ERR_INVALID_LIST;
  if (kind == 6)
    return na_task_graph(m, n, nb, ib, list, count, tasks, task_cap, succ_ptr, succ, succ_cap, ntasks, nedges);
  Problem P{};
  P.m = m;
  P.n = n;
  P.nb = nb;
  P.ib = ib;
  choose_widths(prec, nb, ib, P);
  const std::vector<PanelOp> ops = expand_ops(list, count, m, n);
  Graph g;
  if (kind == 0)
    g = build_factor_graph(ops, m, n, nb, P.w, 0, split_ib_for(prec, P));
  else if (kind >= 3)
    g = build_ls_graph(ops, m, n, nb, P.w, param, 0, kind == 4, split_ib_for(prec, P), kind == 5);
  else
    g = build_apply_graph(ops, m, param, P.wb, kind == 1 ? 1 : 0);
  // successor lists in the order the device copy of the same graph gets them (plans merge their
  // problems' graphs and order them with the tensor-core tile size as the reference)
  if (g_priority_policy == 1 && (kind == 0 || kind >= 3))
    critical_path_priorities(g, (kind == 3 || kind == 5) ? 128 : nb);
  *ntasks = (int64_t)g.tasks.size();
  *nedges = (int64_t)g.succ.size();
  if (!tasks) return HQR_SUCCESS;
  if (task_cap < *ntasks || !succ_ptr || (*nedges > 0 && (!succ || succ_cap < *nedges))) return HQR_ERR_CAPACITY;
  for (size_t q = 0; q < g.tasks.size(); ++q) {
    const Task &t = g.tasks[q];
    const int32_t row[10] = {t.op, t.blk, t.i, t.r, t.k, t.j, t.c0, t.cw, t.trans, t.tgt};
    std::memcpy(tasks + 10 * q, row, sizeof(row));
    succ_ptr[q] = t.succ_begin;
  }
  succ_ptr[g.tasks.size()] = (int64_t)g.succ.size();
  if (!g.succ.empty()) std::memcpy(succ, g.succ.data(), sizeof(int32_t) * g.succ.size());
  return HQR_SUCCESS;
}

int hqr_geqrf(const void *dA, int M, int N, int lda, int prec, int nb, int ib, const hqr_elim_t *list,
              size_t count, hqr_factors **out, void *stream) {
  g_launches = 0;
  if (!dA) return -1;
  if (M < 1) return -2;
  if (N < 1 || N > M) return -3;
  if (lda < M) return -4;
  if (!prec_ok(prec)) return -5;
  if (nb < 8 || nb > 256 || nb % 8 || (prec == HQR_FP32_BF16X3 && nb != tc::NB)) return -6;
  ib = eff_ib(prec, nb, ib);
  if (!valid_tile_sizes(prec, nb, ib)) return -7;
  if (!out) return -10;
  *out = nullptr;
  hqr_factors *F = new (std::nothrow) hqr_factors();
  if (!F) return HQR_ERR_NOMEM;
  F->M = M;
  F->N = N;
  F->nb = nb;
  F->ib = ib;
  F->prec = prec;
  F->m = (M + nb - 1) / nb;
  F->n = (N + nb - 1) / nb;
  F->Mp = F->m * nb;
  F->Np = F->n * nb;
  F->prob.m = F->m;
  F->prob.n = F->n;
  F->prob.nb = nb;
  F->prob.ib = ib;
  choose_widths(prec, nb, ib, F->prob);
  if (list) {
    if (hqr_validate_list(F->m, F->n, list, count) != HQR_SUCCESS) {
      delete F;
      return -8;
    }
    F->list.assign(list, list + count);
  } else {
    size_t cnt = 0;
    hqr_elim_list(F->m, F->n, 4, 1, HQR_GREEDY, HQR_GREEDY, nullptr, 0, &cnt);
    F->list.resize(cnt);
    if (hqr_elim_list(F->m, F->n, 4, 1, HQR_GREEDY, HQR_GREEDY, F->list.data(), cnt, &cnt)) {
      delete F;
      return HQR_ERR_INTERNAL;
    }
  }
  F->ops = expand_ops(F->list.data(), F->list.size(), F->m, F->n);
  Graph g = build_factor_graph(F->ops, F->m, F->n, nb, F->prob.w, 0, split_ib_for(prec, F->prob));
  if (g_priority_policy == 1) critical_path_priorities(g, nb);
  int st = upload_graph(g, F->fg);
  const size_t es = elem_size(prec);
  if (!st) {
    const size_t tsz = (size_t)F->m * F->n * 2 * t_record(prec, nb, ib);
    if (!cuda_ok(cudaMalloc(&F->dA, es * (size_t)F->Mp * F->Np), "cudaMalloc(A)") ||
        !cuda_ok(cudaMalloc(&F->dT, es * tsz), "cudaMalloc(T)") ||
        !cuda_ok(cudaMemset(F->dT, 0, es * tsz), "memset(T)"))
      st = HQR_ERR_NOMEM;
  }
  if (!st) st = push_problem(F);
  if (!st) st = hqr_refactor(F, dA, lda, stream);
  if (st) {
    hqr_factors_free(F);
    return st;
  }
  *out = F;
  return HQR_SUCCESS;
}

int hqr_refactor_async(hqr_factors *F, const void *dA, int lda, void *stream) {
  if (!F) return -1;
  if (!dA) return -2;
  if (lda < F->M) return -3;
  g_launches = 0;
  cudaStream_t s = (cudaStream_t)stream;
  int st = pack_a(F, dA, lda, s);
  if (st) return st;
  return run_graph(F, F->fg, s);
}

int hqr_refactor(hqr_factors *F, const void *dA, int lda, void *stream) {
  int st = hqr_refactor_async(F, dA, lda, stream);
  if (st) return st;
  return read_status(F, (cudaStream_t)stream);
}

int hqr_status(hqr_factors *F, void *stream) {
  if (!F) return -1;
  return read_status(F, (cudaStream_t)stream);
}

int hqr_get_r(const hqr_factors *F, void *dR, int ldr, void *stream) {
  if (!F) return -1;
  if (!dR) return -2;
  if (ldr < F->N) return -3;
  cudaStream_t s = (cudaStream_t)stream;
  const long long total = (long long)F->N * F->N;
  if (F->prec == HQR_FP64)
    unpack_tiles<double><<<grid_for(total), 256, 0, s>>>((const double *)F->dA, F->m, F->nb, (double *)dR, ldr,
                                                         F->N, F->N, 1);
  else
    unpack_tiles<float><<<grid_for(total), 256, 0, s>>>((const float *)F->dA, F->m, F->nb, (float *)dR, ldr, F->N,
                                                        F->N, 1);
  CK(cudaGetLastError());
  return HQR_SUCCESS;
}

int hqr_get_tiles(const hqr_factors *F, void *dOut, int ld, void *stream) {
  if (!F) return -1;
  if (!dOut) return -2;
  if (ld < F->Mp) return -3;
  cudaStream_t s = (cudaStream_t)stream;
  const long long total = (long long)F->Mp * F->Np;
  if (F->prec == HQR_FP64)
    unpack_tiles<double><<<grid_for(total), 256, 0, s>>>((const double *)F->dA, F->m, F->nb, (double *)dOut, ld,
                                                         F->Mp, F->Np, 0);
  else
    unpack_tiles<float><<<grid_for(total), 256, 0, s>>>((const float *)F->dA, F->m, F->nb, (float *)dOut, ld,
                                                        F->Mp, F->Np, 0);
  CK(cudaGetLastError());
  return HQR_SUCCESS;
}

int hqr_get_t(const hqr_factors *F, void *dT, void *stream) {
  if (!F) return -1;
  if (!dT) return -2;
  const size_t es = elem_size(F->prec), rec = (size_t)F->ib * F->nb;
  const size_t stride = t_record(F->prec, F->nb, F->ib), nrec = (size_t)F->m * F->n * 2;
  if (stride == rec)
    CK(cudaMemcpyAsync(dT, F->dT, es * rec * nrec, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  else  // tensor-core records: the T factor follows the split images
    CK(cudaMemcpy2DAsync(dT, es * rec, (const unsigned char *)F->dT + tc::REC_T32, es * stride, es * rec, nrec,
                         cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return HQR_SUCCESS;
}

int hqr_kernel_ms(hqr_factors *F, float *ms) {
  if (!F) return -1;
  if (!ms) return -2;
  if (!F->timed) return HQR_ERR_INTERNAL;
  CK(cudaEventSynchronize(F->ev1));
  CK(cudaEventElapsedTime(ms, F->ev0, F->ev1));
  return HQR_SUCCESS;
}

int hqr_kernel_times(hqr_factors *F, float *ms, int cap, int *count) {
  if (!F) return -1;
  if (!ms) return -2;
  if (cap < 1) return -3;
  if (!count) return -4;
  const int64_t first = std::max(F->ring_read, F->ring_runs - (int64_t)hqr_factors::kRing);
  const int avail = (int)(F->ring_runs - first);
  if (avail > cap) {
    *count = avail;
    return HQR_ERR_CAPACITY;
  }
  *count = avail;
  if (avail == 0) return HQR_SUCCESS;
  const int last = (int)((F->ring_runs - 1) % hqr_factors::kRing);
  CK(cudaEventSynchronize(F->ring[2 * last + 1]));
  for (int q = 0; q < avail; ++q) {
    const int slot = (int)((first + q) % hqr_factors::kRing);
    CK(cudaEventElapsedTime(ms + q, F->ring[2 * slot], F->ring[2 * slot + 1]));
  }
  F->ring_read = F->ring_runs;
  return HQR_SUCCESS;
}

int hqr_trace(hqr_factors *F, int enable, uint64_t *host, size_t cap, size_t *count) {
  if (!F) return -1;
  if (enable == 1) {
    const size_t need = (size_t)F->fg.ntasks;
    if (F->trace_cap < need) {
      cudaFree(F->dtrace);
      F->dtrace = nullptr;
      F->trace_cap = 0;
      if (!cuda_ok(cudaMalloc(&F->dtrace, 3 * sizeof(unsigned long long) * need), "cudaMalloc(trace)"))
        return HQR_ERR_NOMEM;
      F->trace_cap = need;
    }
    return HQR_SUCCESS;
  }
  if (enable == 0) {
    cudaFree(F->dtrace);
    F->dtrace = nullptr;
    F->trace_cap = 0;
    return HQR_SUCCESS;
  }
  if (!count) return -5;
  *count = F->trace_cap;
  if (!F->dtrace) return HQR_SUCCESS;
  if (!host || cap < 3 * F->trace_cap) return HQR_ERR_CAPACITY;
  CK(cudaMemcpy(host, F->dtrace, 3 * sizeof(unsigned long long) * F->trace_cap, cudaMemcpyDeviceToHost));
  return HQR_SUCCESS;
}

int hqr_factors_info(const hqr_factors *F, int *Mp, int *Np, int *m, int *n, int *nb, int *ib,
                     int64_t *ntasks) {
  if (!F) return -1;
  if (Mp) *Mp = F->Mp;
  if (Np) *Np = F->Np;
  if (m) *m = F->m;
  if (n) *n = F->n;
  if (nb) *nb = F->nb;
  if (ib) *ib = F->ib;
  if (ntasks) *ntasks = F->fg.ntasks;
  return HQR_SUCCESS;
}

int hqr_apply_q(hqr_factors *F, int trans, void *dB, int ldb, int nrhs, void *stream) {
  if (!F) return -1;
  if (trans != 0 && trans != 1) return -2;
  if (!dB) return -3;
  if (ldb < F->M) return -4;
  if (nrhs < 0) return -5;
  if (nrhs == 0) return HQR_SUCCESS;
  g_launches = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int wa = F->prob.wb;
  const int nslab = (nrhs + wa - 1) / wa;
  const size_t need = (size_t)F->Mp * nslab * wa;
  const size_t es = elem_size(F->prec);
  if (need > F->bw_cap) {
    CK(cudaStreamSynchronize(s));
    cudaFree(F->dBw);
    F->dBw = nullptr;
    F->bw_cap = 0;
    if (!cuda_ok(cudaMalloc(&F->dBw, es * need), "cudaMalloc(B)")) return HQR_ERR_NOMEM;
    F->bw_cap = need;
    int st = push_problem(F);
    if (st) return st;
  }
  auto key = std::make_pair(trans, nslab);
  auto it = F->ag.find(key);
  if (it == F->ag.end()) {
    Graph g = build_apply_graph(F->ops, F->m, nslab, wa, trans);
    DevGraph d;
    int st = upload_graph(g, d);
    if (st) {
      d.release();
      return st;
    }
    it = F->ag.emplace(key, d).first;
  }
  const long long total = (long long)need;
  if (F->prec == HQR_FP64)
    pack_rhs<double><<<grid_for(total), 256, 0, s>>>((const double *)dB, ldb, F->M, nrhs, (double *)F->dBw, F->m,
                                                     F->nb, wa, total);
  else
    pack_rhs<float><<<grid_for(total), 256, 0, s>>>((const float *)dB, ldb, F->M, nrhs, (float *)F->dBw, F->m,
                                                    F->nb, wa, total);
  CK(cudaGetLastError());
  g_launches += 1;
  int st = run_graph(F, it->second, s);
  if (st) return st;
  const long long tot2 = (long long)F->M * nrhs;
  if (F->prec == HQR_FP64)
    unpack_rhs<double><<<grid_for(tot2), 256, 0, s>>>((const double *)F->dBw, (double *)dB, ldb, F->M, nrhs, F->m,
                                                      F->nb, wa);
  else
    unpack_rhs<float><<<grid_for(tot2), 256, 0, s>>>((const float *)F->dBw, (float *)dB, ldb, F->M, nrhs, F->m,
                                                     F->nb, wa);
  CK(cudaGetLastError());
  g_launches += 1;
  return read_status(F, s);
}

int hqr_gels_qr(const void *dA, int M, int N, int lda, const void *db, int ldb, int nrhs, void *dx, int ldx,
                int prec, int nb, int ib, const hqr_elim_t *list, size_t count, void *stream) {
  if (!db) return -5;
  if (ldb < M) return -6;
  if (nrhs < 1) return -7;
  if (!dx) return -8;
  if (ldx < N) return -9;
  cudaStream_t s = (cudaStream_t)stream;
  hqr_factors *F = nullptr;
  int st = hqr_geqrf(dA, M, N, lda, prec, nb, ib, list, count, &F, stream);
  if (st) return st > 0 ? st : (st <= -5 ? st - 5 : st);
  const size_t es = elem_size(prec);
  void *c = nullptr;
  int *dsing = nullptr;
  int64_t launches = g_launches;
  do {
    if (!cuda_ok(cudaMalloc(&c, es * (size_t)M * nrhs), "cudaMalloc(c)") ||
        !cuda_ok(cudaMalloc(&dsing, sizeof(int)), "cudaMalloc(flag)")) {
      st = HQR_ERR_NOMEM;
      break;
    }
    if (!cuda_ok(cudaMemcpy2DAsync(c, es * M, db, es * ldb, es * M, nrhs, cudaMemcpyDeviceToDevice, s),
                 "copy b") ||
        !cuda_ok(cudaMemsetAsync(dsing, 0, sizeof(int), s), "memset")) {
      st = HQR_ERR_CUDA;
      break;
    }
    st = hqr_apply_q(F, 1, c, M, nrhs, stream);
    launches += g_launches;
    if (st) break;
    for (int i = F->n - 1; i >= 0; --i) {
      const int nbi = std::min(F->nb, N - i * F->nb);
      dim3 gr((i * F->nb + 255) / 256, nrhs);
      if (prec == HQR_FP64) {
        trsv_diag<double><<<nrhs, 256, 0, s>>>((const double *)F->dA, F->m, F->nb, i, nbi, (double *)c, M, dsing);
        if (i > 0) trsv_update<double><<<gr, 256, 0, s>>>((const double *)F->dA, F->m, F->nb, i, nbi, (double *)c, M);
      } else {
        trsv_diag<float><<<nrhs, 256, 0, s>>>((const float *)F->dA, F->m, F->nb, i, nbi, (float *)c, M, dsing);
        if (i > 0) trsv_update<float><<<gr, 256, 0, s>>>((const float *)F->dA, F->m, F->nb, i, nbi, (float *)c, M);
      }
      launches += i > 0 ? 2 : 1;
    }
    if (!cuda_ok(cudaGetLastError(), "trsv") ||
        !cuda_ok(cudaMemcpy2DAsync(dx, es * ldx, c, es * M, es * N, nrhs, cudaMemcpyDeviceToDevice, s),
                 "copy x")) {
      st = HQR_ERR_CUDA;
      break;
    }
    int sing = 0;
    if (!cuda_ok(cudaMemcpyAsync(&sing, dsing, sizeof(int), cudaMemcpyDeviceToHost, s), "flag") ||
        !cuda_ok(cudaStreamSynchronize(s), "sync")) {
      st = HQR_ERR_CUDA;
      break;
    }
    if (sing) st = HQR_ERR_SINGULAR;
  } while (0);
  cudaFree(c);
  cudaFree(dsing);
  hqr_factors_free(F);
  g_launches = launches;
  return st;
}

int hqr_debug_block_task(hqr_factors *F, int64_t task, int extra) {
  if (!F) return -1;
  if (task < 0 || task >= F->fg.ntasks) return -2;
  if (extra < 0) return -3;
  if (F->debug_task >= 0 && F->debug_task != task) return HQR_ERR_INTERNAL;
  if (F->debug_task < 0) {
    // keep the task's true in-degree on the host to restore it later
    CK(cudaMemcpy(&F->debug_base, F->fg.indeg0 + task, sizeof(int), cudaMemcpyDeviceToHost));
    F->debug_task = task;
  }
  const int v = F->debug_base + extra;
  CK(cudaMemcpy(F->fg.indeg0 + task, &v, sizeof(int), cudaMemcpyHostToDevice));
  if (setup_done()) return HQR_ERR_CUDA;
  if (extra == 0) {
    F->debug_task = -1;
    F->debug_base = -1;
  }
  return HQR_SUCCESS;
}

void hqr_factors_free(hqr_factors *F) {
  if (!F) return;
  F->fg.release();
  for (auto &kv : F->ag) kv.second.release();
  cudaFree(F->dA);
  cudaFree(F->dT);
  cudaFree(F->dBw);
  cudaFree(F->dprob);
  cudaFree(F->dtrace);
  if (F->ev0) cudaEventDestroy(F->ev0);
  if (F->ev1) cudaEventDestroy(F->ev1);
  for (cudaEvent_t e : F->ring)
    if (e) cudaEventDestroy(e);
  delete F;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Least-squares plans (one merged task graph for many problems).
namespace {

struct TuneEntry {
  int lm, ln;
  hqr_tile_config_t cfg;
};
std::vector<TuneEntry> g_tuning;

int ilog2(int v) {
  int r = 0;
  while ((v >> (r + 1)) > 0) ++r;
  return r;
}

// Heuristic tile configuration for an M x N problem when no table entry
// applies: tiles large enough for efficient kernels, TS domains of 4 tiles
// (TS updates are the faster kernels, Sec. 5) and greedy trees.
hqr_tile_config_t default_config(int M, int N, int prec) {
  hqr_tile_config_t c;
  c.nb = N <= 48 ? 32 : (N <= 192 || M < 1024 ? 64 : 128);
  c.ib = eff_ib(prec, c.nb, prec == HQR_FP64 ? std::min(16, c.nb / 2) : 16);
  c.a = 4;
  c.p = 1;
  c.low_tree = HQR_GREEDY;
  c.high_tree = HQR_GREEDY;
  return c;
}

hqr_tile_config_t pick_config(int M, int N, int prec, const hqr_tile_config_t *given) {
  hqr_tile_config_t c = default_config(M, N, prec);
  if (given && given->nb > 0) {
    c = *given;
  } else {
    const int lm = ilog2(M), ln = ilog2(N);
    for (const TuneEntry &e : g_tuning)
      if (e.lm == lm && e.ln == ln) {
        c = e.cfg;
        break;
      }
  }
  c.ib = eff_ib(prec, c.nb, c.ib);
  return c;
}

// Per-problem pieces of the preparation and finishing kernels.
struct PrepDesc {
  const void *A;
  long long lda;
  const double *b;
  double *dx;
  void *ws;     // tile workspace
  void *B;      // right-hand-side block (Mp x 1)
  double *x;    // solution vector (Np)
  int M, N, m, n, nb;
  long long off;  // first element of this problem in the flattened index
};

// Flattened per problem: Mp*Np tile elements, then Mp rhs entries, then Np
// entries of x (set to zero). Problems are found by binary search.
template <typename Real>
__global__ void ls_prepare(const PrepDesc *__restrict__ d, int count, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d[mid].off <= e) lo = mid; else hi = mid - 1;
    }
    const PrepDesc &P = d[lo];
    long long q = e - P.off;
    const int nb = P.nb, Mp = P.m * nb, Np = P.n * nb;
    const long long nt = (long long)Mp * Np;
    if (q < nt) {
      const long long nb2 = (long long)nb * nb;
      const long long tile = q / nb2;
      const int w = (int)(q - tile * nb2);
      const int cc = w / nb, rr = w - cc * nb;
      const int row = (int)(tile % P.m) * nb + rr, col = (int)(tile / P.m) * nb + cc;
      ((Real *)P.ws)[q] = (row < P.M && col < P.N) ? ((const Real *)P.A)[(long long)col * P.lda + row] : Real(0);
    } else if ((q -= nt) < Mp) {
      ((Real *)P.B)[q] = q < P.M ? (Real)P.b[q] : Real(0);
    } else {
      q -= Mp;
      P.x[q] = 0.0;
    }
  }
}

__global__ void ls_finish(const PrepDesc *__restrict__ d, int count) {
  for (int pi = blockIdx.x; pi < count; pi += gridDim.x) {
    const PrepDesc &P = d[pi];
    for (int j = threadIdx.x; j < P.N; j += blockDim.x) P.dx[j] = P.x[j];
  }
}

}  // namespace

struct hqr_ls_plan {
  int count = 0, prec = 0, iters = 0;
  int tol_mode = 0;                 // refinement rounds stop at a tolerance (hqr_ls_plan_create_tol)
  double tol = 0.0;
  RefineState *drs = nullptr;       // per-problem refinement state (tol_mode)
  int any_tc = 0;          // some problem runs on the tensor-core kernels
  // Plans with tensor-core and CUDA-core problems run them as two persistent
  // launches side by side: the tensor-core kernel (one CTA per SM) on tc_sms
  // SMs and the CUDA-core kernel (two CTAs per SM) on the others, so that the
  // small problems keep two CTAs per SM. graph holds the tensor-core
  // problems' tasks, graph2 the others'.
  int split = 0;
  DevGraph graph2;
  size_t smem2 = 0;
  int tc_sms = 0;
  double work_tc = 0.0, work_cc = 0.0;  // relative work of the parts (SM share of the next run)
  bool timed_split = false;             // the last run recorded the two kernels' events
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, k0[2] = {nullptr, nullptr}, k1[2] = {nullptr, nullptr};
  std::vector<hqr_tile_config_t> cfg;
  std::vector<Problem> probs;
  std::vector<PrepDesc> prep;
  Problem *dprobs = nullptr;
  PrepDesc *dprep = nullptr;
  void *arena = nullptr;   // tiles, T, rhs blocks (storage precision)
  double *vec = nullptr;   // x, r, g of every problem
  int *dstatus = nullptr;  // per-problem status words
  long long prep_total = 0;
  size_t smem = 0;
  double flops = 0.0;
  DevGraph graph;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraph_t cg = nullptr;
  cudaGraphExec_t cge = nullptr;
  bool ran = false;
  std::vector<int32_t> task_kind;  // op << 24 | problem index, per task (for traces)
  unsigned long long *dtrace = nullptr;
};

namespace {

// out[0] = max_i |d_i|, out[1] = max_i |x_i| over i < n (one block).
__global__ void vec_absmax2(const double *__restrict__ d, const double *__restrict__ x, int n, double *out) {
  __shared__ double sd[256], sx[256];
  double md = 0.0, mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    md = fmax(md, fabs(d[i]));
    mx = fmax(mx, fabs(x[i]));
  }
  sd[threadIdx.x] = md;
  sx[threadIdx.x] = mx;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + h]);
      sx[threadIdx.x] = fmax(sx[threadIdx.x], sx[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sd[0];
    out[1] = sx[0];
  }
}

int plan_enqueue(hqr_ls_plan *P, cudaStream_t s, bool timed) {
  if (P->prec == HQR_FP64)
    ls_prepare<double><<<grid_for(P->prep_total), 256, 0, s>>>(P->dprep, P->count, P->prep_total);
  else
    ls_prepare<float><<<grid_for(P->prep_total), 256, 0, s>>>(P->dprep, P->count, P->prep_total);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(P->dstatus, 0, sizeof(int) * P->count, s));
  if (P->drs) CK(cudaMemsetAsync(P->drs, 0, sizeof(RefineState) * P->count, s));
  for (DevGraph *g : {&P->graph, &P->graph2}) {
    if (!g->ntasks) continue;
    CK(cudaMemcpyAsync(g->indeg, g->indeg0, sizeof(int) * g->ntasks, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(g->slots, g->slots0, sizeof(int) * slot_count(g->ntasks), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(g->ctl, g->ctl0, sizeof(Ctl), cudaMemcpyDeviceToDevice, s));
  }
  auto params = [&](const DevGraph &g, int tc, unsigned long long *trace) {
    EngineParams p{};
    p.tc = tc;
    p.probs = P->dprobs;
    p.tasks = g.tasks;
    p.ntasks = g.ntasks;
    p.succ = g.succ;
    p.indeg = g.indeg;
    p.slots = g.slots;
    p.ctl = g.ctl;
    p.timeout_ns = g_timeout_ns;
    p.trace = trace;
    return p;
  };
  if (timed) CK(cudaEventRecord(P->ev0, s));
  if (!P->split) {
    int st = launch_sched(P->prec, params(P->graph, P->any_tc, P->dtrace), P->smem, s);
    if (st) return st;
  } else {
    // the two parts side by side: tensor-core kernel on s (tc_sms CTAs), CUDA-core kernel on
    // the side stream (two CTAs on each other SM)
    int sms = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (P->tc_sms <= 0) {
      const double w = P->work_tc + P->work_cc;
      P->tc_sms = (int)std::lround(sms * (w > 0 ? P->work_tc / w : 0.5));
    }
    P->tc_sms = std::max(1, std::min(sms - 1, P->tc_sms));
    CK(cudaEventRecord(P->fork, s));
    CK(cudaStreamWaitEvent(P->side, P->fork, 0));
    if (timed) CK(cudaEventRecord(P->k0[0], s));
    int st = launch_sched(P->prec, params(P->graph, 1, P->dtrace), P->smem, s, P->tc_sms);
    if (st) return st;
    if (timed) CK(cudaEventRecord(P->k1[0], s));
    if (timed) CK(cudaEventRecord(P->k0[1], P->side));
    st = launch_sched(P->prec, params(P->graph2, 0, P->dtrace ? P->dtrace + 3 * (size_t)P->graph.ntasks : nullptr),
                      P->smem2, P->side, 2 * (sms - P->tc_sms));
    if (st) return st;
    if (timed) CK(cudaEventRecord(P->k1[1], P->side));
    CK(cudaEventRecord(P->join, P->side));
    CK(cudaStreamWaitEvent(s, P->join, 0));
    P->timed_split = timed;
  }
  if (timed) CK(cudaEventRecord(P->ev1, s));
  ls_finish<<<std::min(P->count, 4096), 256, 0, s>>>(P->dprep, P->count);
  CK(cudaGetLastError());
  return HQR_SUCCESS;
}

}  // namespace

extern "C" {

int hqr_set_tuning(int count, const int *keys, const hqr_tile_config_t *cfgs) {
  if (count < 0) return -1;
  if (count > 0 && (!keys || !cfgs)) return -2;
  g_tuning.clear();
  for (int e = 0; e < count; ++e) g_tuning.push_back({keys[2 * e], keys[2 * e + 1], cfgs[e]});
  return HQR_SUCCESS;
}

}  // extern "C"

namespace {

int plan_create(int count, const hqr_ls_problem_t *probs, const hqr_tile_config_t *cfg, int prec,
                int refine_iters, bool tol_mode, double tol, hqr_ls_plan **plan) {
  *plan = nullptr;
  hqr_ls_plan *P = new (std::nothrow) hqr_ls_plan();
  if (!P) return HQR_ERR_NOMEM;
  P->count = count;
  P->prec = prec;
  P->iters = refine_iters;
  P->tol_mode = tol_mode && refine_iters > 0;
  P->tol = tol;
  const size_t es = elem_size(prec);
  // tile configurations, lists, sizes
  std::vector<size_t> off_tiles(count), off_t(count), off_b(count), off_vec(count);
  size_t arena_elems = 0, vec_elems = 0;
  Graph merged, merged2;  // with split launches: tensor-core problems, the others
  size_t smem = 0;
  for (int q = 0; q < count; ++q) {
    const hqr_ls_problem_t &pr = probs[q];
    if (pr.M < 1 || pr.N < 1 || pr.N > pr.M || pr.lda < pr.M || !pr.dA || !pr.db || !pr.dx) {
      delete P;
      return -2;
    }
    hqr_tile_config_t c = pick_config(pr.M, pr.N, prec, cfg ? &cfg[q] : nullptr);
    if (!valid_tile_sizes(prec, c.nb, c.ib) || c.a < 1 || c.p < 1 || c.low_tree < 0 || c.low_tree > 3 ||
        c.high_tree < 0 || c.high_tree > 3) {
      delete P;
      return -3;
    }
    P->cfg.push_back(c);
    Problem pb{};
    pb.nb = c.nb;
    pb.ib = c.ib;
    pb.m = (pr.M + c.nb - 1) / c.nb;
    pb.n = (pr.N + c.nb - 1) / c.nb;
    choose_widths(prec, c.nb, c.ib, pb);
    drop_t32(prec, pb);
    pb.wb = 1;
    pb.M = pr.M;
    pb.N = pr.N;
    pb.A0 = pr.dA;
    pb.lda0 = pr.lda;
    pb.b = pr.db;
    const size_t Mp = (size_t)pb.m * c.nb, Np = (size_t)pb.n * c.nb;
    off_tiles[q] = arena_elems;
    arena_elems += (Mp * Np + 3) & ~(size_t)3;
    off_t[q] = arena_elems;
    arena_elems += ((size_t)pb.m * pb.n * 2 * t_record(prec, c.nb, c.ib, false) + 3) & ~(size_t)3;
    off_b[q] = arena_elems;
    arena_elems += (Mp + 3) & ~(size_t)3;
    off_vec[q] = vec_elems;
    vec_elems += Np + Mp + Np + 2 * (size_t)atr_chunks(pb.m) * Np + 2 * (size_t)res_chunks(pb.n) * Mp +
                 (size_t)pb.n * c.nb * c.nb + 2 * (size_t)pb.n;
    size_t cnt = 0;
    hqr_elim_list(pb.m, pb.n, c.a, c.p, c.low_tree, c.high_tree, nullptr, 0, &cnt);
    std::vector<hqr_elim_t> lst(cnt);
    if (hqr_elim_list(pb.m, pb.n, c.a, c.p, c.low_tree, c.high_tree, lst.data(), cnt, &cnt)) {
      delete P;
      return HQR_ERR_INTERNAL;
    }
    std::vector<PanelOp> ops = expand_ops(lst.data(), lst.size(), pb.m, pb.n);
    const bool tcp = use_tc(prec, c.nb);
    Graph gq = build_ls_graph(ops, pb.m, pb.n, c.nb, pb.w, refine_iters, q, false, split_ib_for(prec, pb),
                              P->tol_mode != 0);
    append_graph(tcp || !g_split_launch ? merged : merged2, gq);
    if (P->tol_mode) {
      pb.maxit = refine_iters;
      pb.tol = tol;
    }
    if (tcp || !g_split_launch)
      smem = std::max(smem, smem_for(prec, pb));
    else
      P->smem2 = std::max(P->smem2, smem_for(prec, pb));
    if (pb.tc) P->any_tc = 1;
    P->probs.push_back(pb);
    P->flops += 2.0 * pr.M * (double)pr.N * pr.N - 2.0 / 3.0 * (double)pr.N * pr.N * pr.N;
  }
  int st = HQR_SUCCESS;
  if (!cuda_ok(cudaMalloc(&P->arena, es * std::max<size_t>(arena_elems, 1)), "cudaMalloc(arena)") ||
      !cuda_ok(cudaMalloc(&P->vec, sizeof(double) * std::max<size_t>(vec_elems, 1)), "cudaMalloc(vec)") ||
      !cuda_ok(cudaMalloc(&P->dstatus, sizeof(int) * count), "cudaMalloc(status)") ||
      (tol_mode && !cuda_ok(cudaMalloc(&P->drs, sizeof(RefineState) * count), "cudaMalloc(refine state)")) ||
      !cuda_ok(cudaMemset(P->arena, 0, es * std::max<size_t>(arena_elems, 1)), "memset(arena)"))
    st = HQR_ERR_NOMEM;
  if (!st) {
    long long off = 0;
    for (int q = 0; q < count; ++q) {
      Problem &pb = P->probs[q];
      unsigned char *base = (unsigned char *)P->arena;
      pb.A = base + es * off_tiles[q];
      pb.T = base + es * off_t[q];
      pb.B = base + es * off_b[q];
      pb.x = P->vec + off_vec[q];
      pb.r = pb.x + (size_t)pb.n * pb.nb;
      pb.g = pb.r + (size_t)pb.m * pb.nb;
      pb.gp = pb.g + (size_t)pb.n * pb.nb;
      pb.rp = pb.gp + 2 * (size_t)atr_chunks(pb.m) * pb.n * pb.nb;
      pb.rinv = pb.rp + 2 * (size_t)res_chunks(pb.n) * pb.m * pb.nb;
      pb.rn = pb.rinv + (size_t)pb.n * pb.nb * pb.nb;
      pb.status = P->dstatus + q;
      pb.rs = P->drs ? P->drs + q : nullptr;
      PrepDesc d;
      d.A = probs[q].dA;
      d.lda = probs[q].lda;
      d.b = probs[q].db;
      d.dx = probs[q].dx;
      d.ws = pb.A;
      d.B = pb.B;
      d.x = pb.x;
      d.M = pb.M;
      d.N = pb.N;
      d.m = pb.m;
      d.n = pb.n;
      d.nb = pb.nb;
      d.off = off;
      off += (long long)pb.m * pb.nb * pb.n * pb.nb + (long long)pb.m * pb.nb + (long long)pb.n * pb.nb;
      P->prep.push_back(d);
    }
    P->prep_total = off;
    if (!cuda_ok(cudaMalloc(&P->dprobs, sizeof(Problem) * count), "cudaMalloc(probs)") ||
        !cuda_ok(cudaMalloc(&P->dprep, sizeof(PrepDesc) * count), "cudaMalloc(prep)"))
      st = HQR_ERR_NOMEM;
  }
  if (!st && (!cuda_ok(cudaMemcpy(P->dprobs, P->probs.data(), sizeof(Problem) * count, cudaMemcpyHostToDevice),
                       "copy probs") ||
              !cuda_ok(cudaMemcpy(P->dprep, P->prep.data(), sizeof(PrepDesc) * count, cudaMemcpyHostToDevice),
                       "copy prep") ||
              !cuda_ok(cudaEventCreate(&P->ev0), "event") || !cuda_ok(cudaEventCreate(&P->ev1), "event")))
    st = HQR_ERR_CUDA;
  if (!st && !merged2.tasks.empty() && merged.tasks.empty()) {  // no tensor-core problem after all
    merged = std::move(merged2);
    merged2 = Graph();
    smem = P->smem2;
  }
  P->split = !merged2.tasks.empty();
  if (!st) {
    if (g_priority_policy == 1) critical_path_priorities(merged, 128);
    st = upload_graph(merged, P->graph);
  }
  if (!st && P->split) {
    if (g_priority_policy == 1) critical_path_priorities(merged2, 128);
    st = upload_graph(merged2, P->graph2);
    // first SM share: by the QR flops of each part, the tensor-core part's counted at a third
    // (its tiles run about three times faster); rebalanced after every timed run
    double ftc = 0.0, fcc = 0.0;
    for (int q = 0; q < count; ++q) {
      const double f = 2.0 * probs[q].M * (double)probs[q].N * probs[q].N;
      if (P->probs[q].tc) ftc += f; else fcc += f;
    }
    P->work_tc = ftc / 3.0;
    P->work_cc = fcc;
    if (!st && (!cuda_ok(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking), "side stream") ||
                !cuda_ok(cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming), "event") ||
                !cuda_ok(cudaEventCreateWithFlags(&P->join, cudaEventDisableTiming), "event")))
      st = HQR_ERR_CUDA;
    for (int q = 0; q < 2 && !st; ++q)
      if (!cuda_ok(cudaEventCreate(&P->k0[q]), "event") || !cuda_ok(cudaEventCreate(&P->k1[q]), "event"))
        st = HQR_ERR_CUDA;
  }
  P->smem = smem;
  if (st) {
    hqr_ls_plan_free(P);
    return st;
  }
  P->task_kind.resize(merged.tasks.size() + merged2.tasks.size());
  for (size_t t = 0; t < merged.tasks.size(); ++t)
    P->task_kind[t] = ((int32_t)merged.tasks[t].op << 24) | merged.tasks[t].pid;
  for (size_t t = 0; t < merged2.tasks.size(); ++t)
    P->task_kind[merged.tasks.size() + t] = ((int32_t)merged2.tasks[t].op << 24) | merged2.tasks[t].pid;
  *plan = P;
  return HQR_SUCCESS;
}

// Refinement outcome of problem idx (synchronizes s): rounds applied, the
// last applied correction max |d| / max |x| (-1 without refinement), whether
// the tolerance was met, and the first column with a zero diagonal entry of R
// (-1: none; tolerance plans only).
int plan_refine_state(hqr_ls_plan *P, int idx, cudaStream_t s, int *iters, double *rel, int *met, int64_t *sing,
                      int *ncomp = nullptr) {
  *iters = P->iters;
  *rel = -1.0;
  *met = 0;
  *sing = -1;
  if (ncomp) *ncomp = std::min(P->iters, std::max(4, (2 * P->iters + 4) / 5));
  if (!P->drs) return HQR_SUCCESS;
  RefineState h;
  CK(cudaMemcpyAsync(&h, P->drs + idx, sizeof(RefineState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *sing = h.sing ? (int64_t)(~h.sing) : -1;
  if (!P->tol_mode) return HQR_SUCCESS;
  *met = h.met;
  *iters = h.conv ? h.conv : P->iters;
  *rel = *iters > 0 ? h.cval[*iters - 1] : -1.0;
  if (ncomp) {
    *ncomp = 0;
    for (int r = 0; r < *iters; ++r) *ncomp += h.mode[r] != 0;
  }
  return HQR_SUCCESS;
}

}  // namespace

extern "C" {

int hqr_ls_plan_create(int count, const hqr_ls_problem_t *probs, const hqr_tile_config_t *cfg, int prec,
                       int refine_iters, hqr_ls_plan **plan) {
  if (count < 1) return -1;
  if (!probs) return -2;
  if (!prec_ok(prec)) return -4;
  if (refine_iters < 0 || refine_iters > kMaxRounds) return -5;
  if (!plan) return -6;
  return plan_create(count, probs, cfg, prec, refine_iters, false, 0.0, plan);
}

int hqr_ls_plan_create_tol(int count, const hqr_ls_problem_t *probs, const hqr_tile_config_t *cfg, int prec,
                           int max_iter, double tol, hqr_ls_plan **plan) {
  if (count < 1) return -1;
  if (!probs) return -2;
  if (!prec_ok(prec)) return -4;
  if (max_iter < 1 || max_iter > kMaxRounds) return -5;
  if (!(tol >= 0.0)) return -6;
  if (!plan) return -7;
  return plan_create(count, probs, cfg, prec, max_iter, true, tol, plan);
}

int hqr_ls_plan_refine_info(hqr_ls_plan *P, int idx, int *iters, double *rel_correction, int *converged,
                            int *compensated, int64_t *singular_index, void *stream) {
  if (!P) return -1;
  if (idx < 0 || idx >= P->count) return -2;
  int it = 0, met = 0, nc = 0;
  double rel = -1.0;
  int64_t sing = -1;
  const int st = plan_refine_state(P, idx, (cudaStream_t)stream, &it, &rel, &met, &sing, &nc);
  if (st) return st;
  if (iters) *iters = it;
  if (rel_correction) *rel_correction = rel;
  if (converged) *converged = met;
  if (compensated) *compensated = nc;
  if (singular_index) *singular_index = sing;
  return HQR_SUCCESS;
}

int hqr_ls_plan_trace(hqr_ls_plan *P, int enable, uint64_t *host, size_t cap, size_t *count) {
  if (!P) return -1;
  const size_t nt = (size_t)P->graph.ntasks + (size_t)P->graph2.ntasks;
  if (enable == 1) {
    if (!P->dtrace && !cuda_ok(cudaMalloc(&P->dtrace, 3 * sizeof(unsigned long long) * nt), "cudaMalloc(trace)"))
      return HQR_ERR_NOMEM;
    return HQR_SUCCESS;
  }
  if (enable == 0) {
    cudaFree(P->dtrace);
    P->dtrace = nullptr;
    return HQR_SUCCESS;
  }
  if (!count) return -5;
  *count = P->dtrace ? nt : 0;
  if (!P->dtrace) return HQR_SUCCESS;
  if (!host || cap < 4 * nt) return HQR_ERR_CAPACITY;
  std::vector<unsigned long long> tmp(3 * nt);
  CK(cudaMemcpy(tmp.data(), P->dtrace, 3 * sizeof(unsigned long long) * nt, cudaMemcpyDeviceToHost));
  for (size_t t = 0; t < nt; ++t) {
    host[4 * t + 0] = tmp[3 * t + 0];
    host[4 * t + 1] = tmp[3 * t + 1];
    host[4 * t + 2] = tmp[3 * t + 2];
    host[4 * t + 3] = (uint64_t)(uint32_t)P->task_kind[t];
  }
  return HQR_SUCCESS;
}

int hqr_ls_plan_run(hqr_ls_plan *P, void *stream) {
  if (!P) return -1;
  g_launches = 0;
  cudaStream_t s = (cudaStream_t)stream;
  P->ran = true;
  if (P->cge) {  // events around the whole graph: preparation + task kernel + finish
    CK(cudaEventRecord(P->ev0, s));
    CK(cudaGraphLaunch(P->cge, s));
    CK(cudaEventRecord(P->ev1, s));
    g_launches = 3;
    return HQR_SUCCESS;
  }
  if (P->split && P->timed_split && cudaEventQuery(P->k1[1]) == cudaSuccess && cudaEventQuery(P->k1[0]) == cudaSuccess) {
    // SM share from the last timed run: each part's work = its time x its SMs
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, P->k0[0], P->k1[0]) == cudaSuccess &&
        cudaEventElapsedTime(&b, P->k0[1], P->k1[1]) == cudaSuccess && a > 0.f && b > 0.f) {
      int sms = 0, dev = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      P->work_tc = (double)a * P->tc_sms;
      P->work_cc = (double)b * (sms - P->tc_sms);
      P->tc_sms = (int)std::lround(sms * P->work_tc / (P->work_tc + P->work_cc));
    }
  }
  int st = plan_enqueue(P, s, true);
  g_launches += 2;  // preparation and finishing kernels (the task kernels counted at launch)
  return st;
}

int hqr_ls_plan_capture(hqr_ls_plan *P, void *stream) {
  if (!P) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  if (!s) return -2;
  if (P->cge) {
    cudaGraphExecDestroy(P->cge);
    P->cge = nullptr;
  }
  if (P->cg) {
    cudaGraphDestroy(P->cg);
    P->cg = nullptr;
  }
  int grid = 0;  // sets the kernels' shared-memory attributes outside the capture
  int st = ctas_for(P->prec, P->any_tc != 0, P->smem, P->graph.ntasks, &grid);
  if (st) return st;
  if (P->split && (st = ctas_for(P->prec, false, P->smem2, P->graph2.ntasks, &grid))) return st;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  st = plan_enqueue(P, s, false);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  CK(e);
  P->cg = g;
  CK(cudaGraphInstantiate(&P->cge, P->cg, 0));
  return HQR_SUCCESS;
}

int hqr_ls_plan_status(hqr_ls_plan *P, void *stream) {
  if (!P) return -1;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CtlLine c;
  CK(cudaMemcpy(&c, &P->graph.ctl->status, sizeof(CtlLine), cudaMemcpyDeviceToHost));
  if (c.v) return (int)c.v;
  if (P->split) {
    CK(cudaMemcpy(&c, &P->graph2.ctl->status, sizeof(CtlLine), cudaMemcpyDeviceToHost));
    if (c.v) return (int)c.v;
  }
  std::vector<int> stv(P->count);
  CK(cudaMemcpy(stv.data(), P->dstatus, sizeof(int) * P->count, cudaMemcpyDeviceToHost));
  for (int v : stv)
    if (v) return v;
  return HQR_SUCCESS;
}

int hqr_ls_plan_correction(hqr_ls_plan *P, int idx, double *rel, void *stream) {
  if (!P) return -1;
  if (idx < 0 || idx >= P->count) return -2;
  if (!rel) return -3;
  *rel = -1.0;
  if (P->iters == 0) return HQR_SUCCESS;
  if (P->tol_mode) {  // the last applied round's (later rounds may leave scratch vectors behind)
    int it = 0, met = 0;
    int64_t sing = -1;
    return plan_refine_state(P, idx, (cudaStream_t)stream, &it, rel, &met, &sing);
  }
  const Problem &pb = P->probs[idx];
  double *out = nullptr;
  if (!cuda_ok(cudaMalloc(&out, 2 * sizeof(double)), "cudaMalloc(correction)")) return HQR_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  vec_absmax2<<<1, 256, 0, s>>>(pb.g, pb.x, pb.N, out);
  double h[2] = {0.0, 0.0};
  const bool ok = cuda_ok(cudaGetLastError(), "correction kernel") &&
                  cuda_ok(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s), "copy correction") &&
                  cuda_ok(cudaStreamSynchronize(s), "sync correction");
  cudaFree(out);
  if (!ok) return HQR_ERR_CUDA;
  *rel = h[1] > 0.0 ? h[0] / h[1] : (h[0] > 0.0 ? INFINITY : 0.0);
  return HQR_SUCCESS;
}

int hqr_ls_plan_info(hqr_ls_plan *P, int64_t *ntasks, double *qr_flops, float *kernel_ms) {
  if (!P) return -1;
  if (ntasks) *ntasks = P->graph.ntasks + P->graph2.ntasks;
  if (qr_flops) *qr_flops = P->flops;
  if (kernel_ms) {
    *kernel_ms = 0.f;
    if (P->ran) {
      CK(cudaEventSynchronize(P->ev1));
      CK(cudaEventElapsedTime(kernel_ms, P->ev0, P->ev1));
    }
  }
  return HQR_SUCCESS;
}

int hqr_ls_plan_config(const hqr_ls_plan *P, int idx, hqr_tile_config_t *cfg) {
  if (!P) return -1;
  if (idx < 0 || idx >= P->count) return -2;
  if (!cfg) return -3;
  *cfg = P->cfg[idx];
  return HQR_SUCCESS;
}

void hqr_ls_plan_free(hqr_ls_plan *P) {
  if (!P) return;
  P->graph.release();
  P->graph2.release();
  if (P->side) cudaStreamDestroy(P->side);
  for (cudaEvent_t e : {P->fork, P->join, P->k0[0], P->k0[1], P->k1[0], P->k1[1]})
    if (e) cudaEventDestroy(e);
  if (P->cge) cudaGraphExecDestroy(P->cge);
  if (P->cg) cudaGraphDestroy(P->cg);
  cudaFree(P->arena);
  cudaFree(P->vec);
  cudaFree(P->dstatus);
  cudaFree(P->drs);
  cudaFree(P->dprobs);
  cudaFree(P->dprep);
  cudaFree(P->dtrace);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  delete P;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// hqr_gels: one least-squares solve through a plan, with its diagnostics.
namespace {

// Partial sums of b - A x over column chunk blockIdx.y of `cw` columns, one
// thread per row: part[chunk * M + row] (plain FP64 FMAs; a diagnostic).
template <typename Real>
__global__ void diag_resid_part(const Real *__restrict__ A, long long lda, int M, int N, int cw,
                                const double *__restrict__ x, double *__restrict__ part) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= M) return;
  const int c0 = blockIdx.y * cw, c1 = min(N, c0 + cw);
  double s = 0.0;
  for (int c = c0; c < c1; ++c) s = fma((double)A[(long long)c * lda + row], x[c], s);
  part[(size_t)blockIdx.y * M + row] = s;
}

// r = b - (sum of the chunk partials, in chunk order).
__global__ void diag_resid_sum(const double *__restrict__ part, int nch, int M, const double *__restrict__ b,
                               double *__restrict__ r) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= M) return;
  double s = 0.0;
  for (int c = 0; c < nch; ++c) s += part[(size_t)c * M + row];
  r[row] = b[row] - s;
}

// out[col] = sum of squares of column col of A (one warp per column), and
// out[N + col] = (A^T r)_col.
template <typename Real>
__global__ void diag_cols(const Real *__restrict__ A, long long lda, int M, int N, const double *__restrict__ r,
                          double *__restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  const Real *col = A + (long long)warp * lda;
  double ss = 0.0, d = 0.0;
  for (int i = lane; i < M; i += 32) {
    const double a = (double)col[i];
    ss = fma(a, a, ss);
    d = fma(a, r[i], d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if (lane == 0) {
    out[warp] = ss;
    out[N + warp] = d;
  }
}

// One block: out[0] = sum v1^2 (n1 entries of v1: plain squares) ... four
// sums in a fixed order: ||A||_F^2 (column sums), ||A^T r||^2, ||r||^2,
// ||x||^2, ||b||^2.
__global__ void diag_norms(const double *__restrict__ colss, const double *__restrict__ atr, int N,
                           const double *__restrict__ r, const double *__restrict__ b, int M,
                           const double *__restrict__ x, double *__restrict__ out) {
  __shared__ double red[5][256];
  double v[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    v[0] += colss[i];
    v[1] = fma(atr[i], atr[i], v[1]);
    v[3] = fma(x[i], x[i], v[3]);
  }
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    v[2] = fma(r[i], r[i], v[2]);
    v[4] = fma(b[i], b[i], v[4]);
  }
  for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = red[threadIdx.x][0];
}

// ||b - A x||, ||A||_F, ||x||, ||b|| and ||A^T (b - A x)|| of a solved
// problem (plain FP64 on the device): the backward error and the
// normal-equation residual of hqr_gels_info.
int gels_diagnostics(const void *dA, int M, int N, int lda, const double *db, const double *dx, int prec,
                     cudaStream_t s, double *bwd, double *nres) {
  const int cw = 256, nch = (N + cw - 1) / cw;
  double *buf = nullptr;
  const size_t need = (size_t)nch * M + M + 2 * (size_t)N + 8;
  if (!cuda_ok(cudaMalloc(&buf, sizeof(double) * need), "cudaMalloc(gels diagnostics)")) return HQR_ERR_NOMEM;
  double *part = buf, *r = part + (size_t)nch * M, *cols = r + M, *out = cols + 2 * (size_t)N;
  const dim3 g1((M + 255) / 256, nch);
  if (prec == HQR_FP64) {
    diag_resid_part<double><<<g1, 256, 0, s>>>((const double *)dA, lda, M, N, cw, dx, part);
  } else {
    diag_resid_part<float><<<g1, 256, 0, s>>>((const float *)dA, lda, M, N, cw, dx, part);
  }
  diag_resid_sum<<<(M + 255) / 256, 256, 0, s>>>(part, nch, M, db, r);
  if (prec == HQR_FP64)
    diag_cols<double><<<(N * 32 + 255) / 256, 256, 0, s>>>((const double *)dA, lda, M, N, r, cols);
  else
    diag_cols<float><<<(N * 32 + 255) / 256, 256, 0, s>>>((const float *)dA, lda, M, N, r, cols);
  diag_norms<<<1, 256, 0, s>>>(cols, cols + N, N, r, db, M, dx, out);
  double h[5] = {0, 0, 0, 0, 0};
  const bool ok = cuda_ok(cudaGetLastError(), "gels diagnostics") &&
                  cuda_ok(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s), "copy diagnostics") &&
                  cuda_ok(cudaStreamSynchronize(s), "sync diagnostics");
  cudaFree(buf);
  if (!ok) return HQR_ERR_CUDA;
  const double na = std::sqrt(h[0]), natr = std::sqrt(h[1]), nr = std::sqrt(h[2]), nx = std::sqrt(h[3]),
               nbv = std::sqrt(h[4]);
  *bwd = (na * nx + nbv) > 0.0 ? nr / (na * nx + nbv) : 0.0;
  *nres = (na * nr) > 0.0 ? natr / (na * nr) : 0.0;
  return HQR_SUCCESS;
}

}  // namespace

extern "C" int hqr_gels(const void *dA, int M, int N, int lda, const double *db, double *dx, int prec, double tol,
                        int max_iter, hqr_gels_info *info, void *stream) {
  if (!dA) return -1;
  if (M < 1) return -2;
  if (N < 1 || N > M) return -3;
  if (lda < M) return -4;
  if (!db) return -5;
  if (!dx) return -6;
  if (!prec_ok(prec)) return -7;
  if (!(tol >= 0.0)) return -8;
  if (max_iter < 0 || max_iter > kMaxRounds) return -9;
  cudaStream_t s = (cudaStream_t)stream;
  hqr_ls_problem_t pr;
  pr.M = M;
  pr.N = N;
  pr.dA = dA;
  pr.lda = lda;
  pr.db = db;
  pr.dx = dx;
  hqr_ls_plan *P = nullptr;
  int st = plan_create(1, &pr, nullptr, prec, max_iter, true, tol, &P);
  if (st) return st;
  st = hqr_ls_plan_run(P, stream);
  const int64_t launches = g_launches;
  if (!st) st = hqr_ls_plan_status(P, stream);
  hqr_gels_info inf;
  inf.iters = 0;
  inf.converged = max_iter == 0 ? 1 : 0;
  inf.rel_correction = -1.0;
  inf.backward_error = -1.0;
  inf.normal_residual = -1.0;
  inf.singular_index = -1;
  if (st == HQR_SUCCESS || st == HQR_ERR_NOCONV || st == HQR_ERR_SINGULAR) {
    int it = 0, met = 0;
    double rel = -1.0;
    int64_t sing = -1;
    const int s2 = plan_refine_state(P, 0, s, &it, &rel, &met, &sing);
    if (s2) {
      st = s2;
    } else {
      if (max_iter > 0) {
        inf.iters = it;
        inf.converged = met;
        inf.rel_correction = rel;
      }
      inf.singular_index = sing;
      if (st != HQR_ERR_SINGULAR) {
        const int s3 = gels_diagnostics(dA, M, N, lda, db, dx, prec, s, &inf.backward_error, &inf.normal_residual);
        if (s3) st = s3;
      }
    }
  }
  hqr_ls_plan_free(P);
  g_launches = launches + 5;
  if (info) *info = inf;
  return st;
}

// ---------------------------------------------------------------------------
// Measured autotuner for least-squares plans.
namespace {

// Unit-cost model of the factorization graph of an m x n tile matrix under a
// tile configuration: critical path and total work (hqr_critical_path).
int config_cost(int m, int n, const hqr_tile_config_t &c, int prec, double *cp, double *work) {
  size_t cnt = 0;
  if (hqr_elim_list(m, n, c.a, c.p, c.low_tree, c.high_tree, nullptr, 0, &cnt) != HQR_ERR_CAPACITY && cnt) return 1;
  std::vector<hqr_elim_t> lst(cnt);
  if (cnt && hqr_elim_list(m, n, c.a, c.p, c.low_tree, c.high_tree, lst.data(), cnt, &cnt)) return 1;
  Problem pb{};
  pb.m = m;
  pb.n = n;
  pb.nb = c.nb;
  pb.ib = eff_ib(prec, c.nb, c.ib);
  choose_widths(prec, c.nb, pb.ib, pb);
  const Graph g = build_factor_graph(expand_ops(lst.data(), lst.size(), m, n), m, n, c.nb, pb.w, 0,
                                     split_ib_for(prec, pb));
  *cp = critical_path_length(g, c.nb);
  *work = total_cost(g, c.nb);
  return 0;
}

// Uniform(-1, 1) entries from a counter-based hash (SplitMix64 finaliser);
// only used to time candidate configurations.
template <typename Real>
__global__ void fill_uniform(Real *x, long long n, unsigned long long seed) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[e] = (Real)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

}  // namespace

extern "C" int hqr_critical_path(int m, int n, int nb, int ib, int prec, const hqr_elim_t *list, size_t count,
                                 double *critical_path, double *work) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (!prec_ok(prec)) return -5;
  if (nb < 8 || nb > 256 || nb % 8 || (prec == HQR_FP32_BF16X3 && nb != tc::NB)) return -3;
  ib = eff_ib(prec, nb, ib);
  if (!valid_tile_sizes(prec, nb, ib)) return -4;
  if (!list && count) return -6;
  if (!critical_path || !work) return -8;
  if (hqr_validate_list(m, n, list, count) != HQR_SUCCESS) return HQR_ERR_INVALID_LIST;
  Problem pb{};
  pb.m = m;
  pb.n = n;
  pb.nb = nb;
  pb.ib = ib;
  choose_widths(prec, nb, ib, pb);
  const Graph g = build_factor_graph(expand_ops(list, count, m, n), m, n, nb, pb.w, 0, split_ib_for(prec, pb));
  *critical_path = critical_path_length(g, nb);
  *work = total_cost(g, nb);
  return HQR_SUCCESS;
}

extern "C" int hqr_autotune(int count, const int *Ms, const int *Ns, int prec, int refine_iters, int reps,
                            int *keys_out, hqr_tile_config_t *cfg_out, int cap, int *nout, void *stream) {
  if (count < 1) return -1;
  if (!Ms) return -2;
  if (!Ns) return -3;
  if (!prec_ok(prec)) return -4;
  if (reps < 1) return -6;
  if (!nout) return -10;
  cudaStream_t s = (cudaStream_t)stream;
  // representative shape per class: geometric mean of its members
  std::map<std::pair<int, int>, std::pair<double, double>> acc;
  std::map<std::pair<int, int>, int> cnt;
  for (int q = 0; q < count; ++q) {
    if (Ms[q] < Ns[q] || Ns[q] < 1) return -2;
    auto key = std::make_pair(ilog2(Ms[q]), ilog2(Ns[q]));
    acc[key].first += std::log((double)Ms[q]);
    acc[key].second += std::log((double)Ns[q]);
    cnt[key] += 1;
  }
  const size_t es = elem_size(prec);
  std::vector<int> keys;
  std::vector<hqr_tile_config_t> best_cfgs;
  for (auto &kv : acc) {
    const int c = cnt[kv.first];
    int M = (int)std::lround(std::exp(kv.second.first / c));
    int N = (int)std::lround(std::exp(kv.second.second / c));
    N = std::max(1, std::min(N, M));
    // workspaces for `reps` copies of the class shape
    void *A = nullptr;
    double *bx = nullptr;
    if (!cuda_ok(cudaMalloc(&A, es * (size_t)M * N * reps), "cudaMalloc(tune A)") ||
        !cuda_ok(cudaMalloc(&bx, sizeof(double) * ((size_t)M + N) * reps), "cudaMalloc(tune b)")) {
      cudaFree(A);
      return HQR_ERR_NOMEM;
    }
    const long long na = (long long)M * N * reps;
    if (prec == HQR_FP64)
      fill_uniform<double><<<grid_for(na), 256, 0, s>>>((double *)A, na, 12345ull + M);
    else
      fill_uniform<float><<<grid_for(na), 256, 0, s>>>((float *)A, na, 12345ull + M);
    fill_uniform<double><<<grid_for((long long)M * reps), 256, 0, s>>>(bx, (long long)M * reps, 777ull + N);
    std::vector<hqr_ls_problem_t> probs(reps);
    for (int r = 0; r < reps; ++r) {
      probs[r].M = M;
      probs[r].N = N;
      probs[r].dA = (const unsigned char *)A + es * (size_t)M * N * r;
      probs[r].lda = M;
      probs[r].db = bx + (size_t)M * r;
      probs[r].dx = bx + (size_t)M * reps + (size_t)N * r;
    }
    std::vector<hqr_tile_config_t> cands;
    for (int nb : {32, 64, 128}) {
      if (nb > 32 && nb / 2 >= N) continue;  // no tile much wider than the matrix
      const int ib = eff_ib(prec, nb, 16);
      const int mtiles = (M + nb - 1) / nb;
      for (int a : {1, 4, 16}) {
        if (a > 1 && a >= 2 * mtiles) continue;
        cands.push_back({nb, ib, a, 1, HQR_GREEDY, HQR_GREEDY});
      }
      cands.push_back({nb, ib, mtiles, 1, HQR_FLAT, HQR_GREEDY});
    }
    float best = 1e30f;
    hqr_tile_config_t best_cfg = default_config(M, N, prec);
    auto try_config = [&](const hqr_tile_config_t &cf) {
      if (!valid_tile_sizes(prec, cf.nb, cf.ib)) return;
      std::vector<hqr_tile_config_t> cfv(reps, cf);
      hqr_ls_plan *P = nullptr;
      int st = hqr_ls_plan_create(reps, probs.data(), cfv.data(), prec, refine_iters, &P);
      if (st) return;
      float ms = 0.f, tot = 0.f;
      bool ok = hqr_ls_plan_run(P, stream) == HQR_SUCCESS;  // warm-up
      for (int it = 0; ok && it < 2; ++it) {
        ok = hqr_ls_plan_run(P, stream) == HQR_SUCCESS && hqr_ls_plan_info(P, nullptr, nullptr, &ms) == 0;
        tot += ms;
      }
      if (ok && hqr_ls_plan_status(P, stream) == HQR_SUCCESS && tot < best) {
        best = tot;
        best_cfg = cf;
      }
      hqr_ls_plan_free(P);
    };
    // stage 1: tile size, TS domain size and low-level tree (one virtual domain)
    for (const hqr_tile_config_t &cf : cands) try_config(cf);
    // stage 2: virtual domains p and the high-level tree for the stage-1 winner. The
    // candidates are ranked by a unit-cost model of the factorization graph (Sec. 2
    // weights): the larger of its critical path and its work spread over the resident
    // CTAs (the reps problems run at once); only the best few are timed.
    {
      const hqr_tile_config_t c1 = best_cfg;
      const int mt = (M + c1.nb - 1) / c1.nb, nt = (N + c1.nb - 1) / c1.nb;
      int sms = 152;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
      const double workers = 2.0 * sms;
      std::vector<std::pair<double, hqr_tile_config_t>> ranked;
      for (int p : {2, 4, 8, 16}) {
        if (2 * p > mt) continue;
        for (int high : {HQR_GREEDY, HQR_FIBONACCI, HQR_BINARY, HQR_FLAT}) {
          hqr_tile_config_t cf = c1;
          cf.p = p;
          cf.high_tree = high;
          double cp = 0.0, work = 0.0;
          if (config_cost(mt, nt, cf, prec, &cp, &work)) continue;
          ranked.push_back({std::max(cp, reps * work / workers), cf});
        }
      }
      std::stable_sort(ranked.begin(), ranked.end(),
                       [](const std::pair<double, hqr_tile_config_t> &a, const std::pair<double, hqr_tile_config_t> &b) {
                         return a.first < b.first;
                       });
      for (size_t q = 0; q < ranked.size() && q < 3; ++q) try_config(ranked[q].second);
    }
    cudaFree(A);
    cudaFree(bx);
    keys.push_back(kv.first.first);
    keys.push_back(kv.first.second);
    best_cfgs.push_back(best_cfg);
  }
  *nout = (int)best_cfgs.size();
  int st = hqr_set_tuning((int)best_cfgs.size(), keys.data(), best_cfgs.data());
  if (st) return st;
  if (keys_out && cfg_out && cap >= (int)best_cfgs.size()) {
    std::memcpy(keys_out, keys.data(), sizeof(int) * keys.size());
    std::memcpy(cfg_out, best_cfgs.data(), sizeof(hqr_tile_config_t) * best_cfgs.size());
  }
  return HQR_SUCCESS;
}

// ---------------------------------------------------------------------------
// Least-squares server: continuous batching on a resident task kernel.
namespace {

// First-fit allocator over [0, cap) (units are the caller's).
class RangeAlloc {
 public:
  void init(size_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
    used_ = 0;
  }
  bool alloc(size_t n, size_t &off) {
    if (n == 0) n = 1;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        off = it->first;
        const size_t rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    if (n == 0) n = 1;
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct CachedGraph {
  Graph g;
  std::vector<int> init;  // tasks with no inputs
};

size_t pow2_at_least(size_t v) {
  size_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

struct hqr_server {
  hqr_server_opts o{};
  size_t es = 0;
  Task *tasks = nullptr;
  int *succ = nullptr, *indeg = nullptr, *initlist = nullptr, *slots = nullptr;
  Ctl *ctl = nullptr;
  ServeCtl *sc = nullptr;
  InboxEntry *inbox = nullptr;
  Problem *probs = nullptr;
  int *req_done = nullptr, *req_total = nullptr, *dstatus = nullptr;
  long long *req_seq = nullptr;
  long long *comp_host = nullptr, *comp_dev = nullptr;
  unsigned char *arena = nullptr;
  int ring_cap = 0, inbox_cap = 0;
  RangeAlloc arena_alloc, task_alloc, edge_alloc;
  std::vector<int> free_slots;
  struct Live {
    long long seq = -1;
    size_t a_off = 0, a_n = 0, t_off = 0, t_n = 0, e_off = 0, e_n = 0;
    bool live = false;
  };
  std::vector<Live> live;
  std::map<std::vector<int>, CachedGraph> cache;
  unsigned inbox_tail = 0;
  long long next_seq = 1;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  bool running = false;
  size_t smem = 0;
  int64_t submitted = 0, completed = 0;
};

namespace {

void server_release(hqr_server *S) {
  cudaFree(S->tasks);
  cudaFree(S->succ);
  cudaFree(S->indeg);
  cudaFree(S->initlist);
  cudaFree(S->slots);
  cudaFree(S->ctl);
  cudaFree(S->sc);
  cudaFree(S->inbox);
  cudaFree(S->probs);
  cudaFree(S->req_done);
  cudaFree(S->req_total);
  cudaFree(S->req_seq);
  cudaFree(S->dstatus);
  cudaFree(S->arena);
  if (S->comp_host) cudaFreeHost(S->comp_host);
  if (S->kstream) cudaStreamDestroy(S->kstream);
  if (S->cstream) cudaStreamDestroy(S->cstream);
}

// Largest shared memory any request configuration of the server may need.
size_t server_smem(int prec) {
  size_t m = 0;
  for (int nb : {32, 64, 128})
    for (int ib0 : {8, 16, 32}) {
      const int ib = eff_ib(prec, nb, ib0);
      if (!valid_tile_sizes(prec, nb, ib)) continue;
      Problem pb{};
      pb.nb = nb;
      pb.ib = ib;
      choose_widths(prec, nb, ib, pb);
      pb.wb = 1;
      m = std::max(m, smem_for(prec, pb));
    }
  return m;
}

}  // namespace

extern "C" {

int hqr_server_create(const hqr_server_opts *o, hqr_server **out) {
  if (!o) return -1;
  if (!out) return -2;
  *out = nullptr;
  if (!prec_ok(o->prec)) return -1;
  if (o->refine_iters < 0 || o->max_live < 1 || o->task_pool < 1024 || o->edge_pool < 1024 || o->hbm_budget < 1)
    return -1;
  hqr_server *S = new (std::nothrow) hqr_server();
  if (!S) return HQR_ERR_NOMEM;
  S->o = *o;
  S->es = elem_size(o->prec);
  const size_t TP = (size_t)o->task_pool, EP = (size_t)o->edge_pool, L = (size_t)o->max_live;
  S->ring_cap = (int)pow2_at_least(TP / kShards + L + 64);
  S->inbox_cap = (int)pow2_at_least(2 * L);
  const size_t nslots = (size_t)kServeQueues * kShards * S->ring_cap;
  int st = HQR_SUCCESS;
  if (!cuda_ok(cudaMalloc(&S->tasks, sizeof(Task) * TP), "server tasks") ||
      !cuda_ok(cudaMalloc(&S->succ, sizeof(int) * EP), "server succ") ||
      !cuda_ok(cudaMalloc(&S->indeg, sizeof(int) * TP), "server indeg") ||
      !cuda_ok(cudaMalloc(&S->initlist, sizeof(int) * TP), "server init") ||
      !cuda_ok(cudaMalloc(&S->slots, sizeof(int) * nslots), "server slots") ||
      !cuda_ok(cudaMalloc(&S->ctl, sizeof(Ctl)), "server ctl") ||
      !cuda_ok(cudaMalloc(&S->sc, sizeof(ServeCtl)), "server sc") ||
      !cuda_ok(cudaMalloc(&S->inbox, sizeof(InboxEntry) * S->inbox_cap), "server inbox") ||
      !cuda_ok(cudaMalloc(&S->probs, sizeof(Problem) * L), "server probs") ||
      !cuda_ok(cudaMalloc(&S->req_done, sizeof(int) * L), "server done") ||
      !cuda_ok(cudaMalloc(&S->req_total, sizeof(int) * L), "server total") ||
      !cuda_ok(cudaMalloc(&S->req_seq, sizeof(long long) * L), "server seq") ||
      !cuda_ok(cudaMalloc(&S->dstatus, sizeof(int) * L), "server status") ||
      !cuda_ok(cudaMalloc(&S->arena, o->hbm_budget), "server arena") ||
      !cuda_ok(cudaHostAlloc(&S->comp_host, sizeof(long long) * L, cudaHostAllocMapped), "server comp") ||
      !cuda_ok(cudaHostGetDevicePointer(&S->comp_dev, S->comp_host, 0), "server comp ptr") ||
      !cuda_ok(cudaMemset(S->slots, 0, sizeof(int) * nslots), "memset slots") ||
      !cuda_ok(cudaMemset(S->ctl, 0, sizeof(Ctl)), "memset ctl") ||
      !cuda_ok(cudaMemset(S->sc, 0, sizeof(ServeCtl)), "memset sc") ||
      !cuda_ok(cudaMemset(S->req_done, 0, sizeof(int) * L), "memset done") ||
      !cuda_ok(cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking), "stream") ||
      !cuda_ok(cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking), "stream"))
    st = HQR_ERR_NOMEM;
  if (!st && setup_done()) st = HQR_ERR_CUDA;  // the fills above land before the kernel or a submission runs
  if (st) {
    server_release(S);
    delete S;
    return st;
  }
  for (size_t q = 0; q < L; ++q) S->comp_host[q] = -1;
  S->arena_alloc.init(o->hbm_budget / 256);
  S->task_alloc.init(TP);
  S->edge_alloc.init(EP);
  S->live.resize(L);
  for (int q = (int)L - 1; q >= 0; --q) S->free_slots.push_back(q);
  S->smem = server_smem(o->prec);
  *out = S;
  return HQR_SUCCESS;
}

// Relaunch the resident kernel if it left (idle exit) while work is owed.
int server_ensure_running(hqr_server *S);

int hqr_server_start(hqr_server *S) {
  if (!S) return -1;
  if (S->running && cudaStreamQuery(S->kstream) == cudaErrorNotReady) return HQR_SUCCESS;
  ServeParams sp{};
  sp.e.tc = S->o.prec == HQR_FP32_BF16X3;
  sp.e.probs = S->probs;
  sp.e.tasks = S->tasks;
  sp.e.ntasks = (int)S->o.task_pool;
  sp.e.succ = S->succ;
  sp.e.indeg = S->indeg;
  sp.e.slots = S->slots;
  sp.e.ctl = S->ctl;
  sp.e.timeout_ns = g_timeout_ns;
  sp.e.trace = nullptr;
  sp.sc = S->sc;
  sp.inbox = S->inbox;
  sp.inbox_cap = S->inbox_cap;
  sp.initlist = S->initlist;
  sp.req_done = S->req_done;
  sp.req_total = S->req_total;
  sp.req_seq = S->req_seq;
  sp.comp = S->comp_dev;
  sp.ring_cap = S->ring_cap;
  const bool tcs = S->o.prec == HQR_FP32_BF16X3;
  const void *k = S->o.prec == HQR_FP64
                      ? (const void *)hqr_serve<double, false>
                      : (tcs ? (const void *)hqr_serve<float, true> : (const void *)hqr_serve<float, false>);
  int dev = 0, sms = 0, per_sm = 0;
  CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S->smem));
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, S->smem));
  if (per_sm < 1) return HQR_ERR_CUDA;
  CK(cudaStreamSynchronize(S->cstream));
  if (S->o.prec == HQR_FP64)
    hqr_serve<double, false><<<sms * per_sm, NT, S->smem, S->kstream>>>(sp);
  else if (tcs)
    hqr_serve<float, true><<<sms * per_sm, NT, S->smem, S->kstream>>>(sp);
  else
    hqr_serve<float, false><<<sms * per_sm, NT, S->smem, S->kstream>>>(sp);
  CK(cudaGetLastError());
  S->running = true;
  return HQR_SUCCESS;
}

int server_ensure_running(hqr_server *S) {
  if (!S->running) return HQR_SUCCESS;
  const cudaError_t q = cudaStreamQuery(S->kstream);
  if (q == cudaErrorNotReady) return HQR_SUCCESS;
  CK(q);
  CtlLine stl;
  CK(cudaMemcpy(&stl, &S->ctl->status, sizeof(CtlLine), cudaMemcpyDeviceToHost));
  if (stl.v) return (int)stl.v;
  S->running = false;
  return hqr_server_start(S);
}

int hqr_server_submit(hqr_server *S, const hqr_ls_problem_t *pr, int64_t *ticket) {
  if (!S) return -1;
  if (!pr || pr->M < 1 || pr->N < 1 || pr->N > pr->M || pr->lda < pr->M || !pr->dA || !pr->db || !pr->dx)
    return -2;
  if (!ticket) return -3;
  if (!S->running) return HQR_ERR_INTERNAL;
  const int prec = S->o.prec;
  hqr_tile_config_t c = pick_config(pr->M, pr->N, prec, nullptr);
  if (c.nb > 128) c.nb = 128;
  if (!valid_tile_sizes(prec, c.nb, c.ib)) c = default_config(pr->M, pr->N, prec);
  Problem pb{};
  pb.nb = c.nb;
  pb.ib = c.ib;
  pb.m = (pr->M + c.nb - 1) / c.nb;
  pb.n = (pr->N + c.nb - 1) / c.nb;
  choose_widths(prec, c.nb, c.ib, pb);
  drop_t32(prec, pb);
  pb.wb = 1;
  // graph of this shape and configuration (cached)
  std::vector<int> key = {pr->M, pr->N, c.nb, c.ib, c.a, c.p, c.low_tree, c.high_tree};
  auto it = S->cache.find(key);
  if (it == S->cache.end()) {
    size_t cnt = 0;
    hqr_elim_list(pb.m, pb.n, c.a, c.p, c.low_tree, c.high_tree, nullptr, 0, &cnt);
    std::vector<hqr_elim_t> lst(cnt);
    if (hqr_elim_list(pb.m, pb.n, c.a, c.p, c.low_tree, c.high_tree, lst.data(), cnt, &cnt))
      return HQR_ERR_INTERNAL;
    CachedGraph cg;
    cg.g = build_ls_graph(expand_ops(lst.data(), lst.size(), pb.m, pb.n), pb.m, pb.n, c.nb, pb.w,
                          S->o.refine_iters, 0, true, split_ib_for(prec, pb));
    if (g_priority_policy == 1) critical_path_priorities(cg.g, c.nb);
    for (size_t t = 0; t < cg.g.tasks.size(); ++t)
      if (cg.g.indeg[t] == 0) cg.init.push_back((int)t);
    if (S->cache.size() > 4096) S->cache.clear();
    it = S->cache.emplace(key, std::move(cg)).first;
  }
  const CachedGraph &cg = it->second;
  const size_t nt = cg.g.tasks.size(), ne = std::max<size_t>(cg.g.succ.size(), 1);
  const size_t Mp = (size_t)pb.m * c.nb, Np = (size_t)pb.n * c.nb, es = S->es;
  auto r256 = [](size_t b) { return (b + 255) / 256; };
  const size_t a_tiles = r256(es * Mp * Np), a_t = r256(es * (size_t)pb.m * pb.n * 2 * t_record(prec, c.nb, c.ib, false)),
               a_b = r256(es * Mp), a_r = r256(8 * Mp), a_g = r256(8 * Np),
               a_gp = r256(16 * (size_t)atr_chunks(pb.m) * Np), a_rp = r256(16 * (size_t)res_chunks(pb.n) * Mp),
               a_ri = r256(8 * (size_t)pb.n * c.nb * c.nb);
  const size_t a_units = a_tiles + a_t + a_b + a_r + a_g + a_gp + a_rp + a_ri;
  if (a_units * 256 > S->o.hbm_budget || nt > (size_t)S->o.task_pool || ne > (size_t)S->o.edge_pool)
    return HQR_ERR_BUDGET;
  if (S->free_slots.empty()) return HQR_ERR_BUSY;
  size_t a_off = 0, t_off = 0, e_off = 0;
  if (!S->arena_alloc.alloc(a_units, a_off)) return HQR_ERR_BUSY;
  if (!S->task_alloc.alloc(nt, t_off)) {
    S->arena_alloc.release(a_off, a_units);
    return HQR_ERR_BUSY;
  }
  if (!S->edge_alloc.alloc(ne, e_off)) {
    S->arena_alloc.release(a_off, a_units);
    S->task_alloc.release(t_off, nt);
    return HQR_ERR_BUSY;
  }
  const int slot = S->free_slots.back();
  S->free_slots.pop_back();
  // patched copies: tasks name the slot, successors are global pool ids
  std::vector<Task> tk(cg.g.tasks);
  for (Task &t : tk) {
    t.pid = slot;
    t.succ_begin += (int32_t)e_off;
    t.succ_end += (int32_t)e_off;
  }
  std::vector<int> sc(cg.g.succ);
  for (int &v : sc) v += (int)t_off;
  std::vector<int> init(cg.init);
  for (int &v : init) v += (int)t_off;
  unsigned char *base = S->arena + a_off * 256;
  pb.A = base;
  pb.T = base + a_tiles * 256;
  pb.B = base + (a_tiles + a_t) * 256;
  pb.r = (double *)(base + (a_tiles + a_t + a_b) * 256);
  pb.g = (double *)(base + (a_tiles + a_t + a_b + a_r) * 256);
  pb.gp = (double *)(base + (a_tiles + a_t + a_b + a_r + a_g) * 256);
  pb.rp = (double *)(base + (a_tiles + a_t + a_b + a_r + a_g + a_gp) * 256);
  pb.rinv = (double *)(base + (a_tiles + a_t + a_b + a_r + a_g + a_gp + a_rp) * 256);
  pb.x = pr->dx;
  pb.M = pr->M;
  pb.N = pr->N;
  pb.A0 = pr->dA;
  pb.lda0 = pr->lda;
  pb.b = pr->db;
  pb.status = S->dstatus + slot;
  const long long seq = S->next_seq++;
  const int total = (int)nt, zero = 0;
  S->comp_host[slot] = -1;
  InboxEntry en{slot, (int)t_off, (int)init.size(), (int)nt};
  cudaStream_t s = S->cstream;
  const unsigned new_tail = S->inbox_tail + 1;
  CK(cudaMemcpyAsync(S->tasks + t_off, tk.data(), sizeof(Task) * nt, cudaMemcpyHostToDevice, s));
  if (!cg.g.succ.empty())
    CK(cudaMemcpyAsync(S->succ + e_off, sc.data(), sizeof(int) * sc.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->indeg + t_off, cg.g.indeg.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->initlist + t_off, init.data(), sizeof(int) * init.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->probs + slot, &pb, sizeof(Problem), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->req_total + slot, &total, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->req_done + slot, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->req_seq + slot, &seq, sizeof(long long), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->dstatus + slot, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S->inbox + (S->inbox_tail & (unsigned)(S->inbox_cap - 1)), &en, sizeof(InboxEntry),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(&S->sc->inbox_tail.v, &new_tail, sizeof(unsigned), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the staged host copies above are stack / temporary buffers
  S->inbox_tail = new_tail;
  {
    const int rs = server_ensure_running(S);
    if (rs) return rs;
  }
  hqr_server::Live &lv = S->live[slot];
  lv.seq = seq;
  lv.a_off = a_off;
  lv.a_n = a_units;
  lv.t_off = t_off;
  lv.t_n = nt;
  lv.e_off = e_off;
  lv.e_n = ne;
  lv.live = true;
  S->submitted += 1;
  *ticket = seq;
  return HQR_SUCCESS;
}

int hqr_server_poll(hqr_server *S, int64_t *done, int cap, int *count) {
  if (!S) return -1;
  if (!count) return -4;
  int n = 0;
  for (size_t slot = 0; slot < S->live.size(); ++slot) {
    hqr_server::Live &lv = S->live[slot];
    if (!lv.live) continue;
    const long long c = *(volatile long long *)&S->comp_host[slot];
    if (c != lv.seq) continue;
    if (done && n < cap) done[n] = lv.seq;
    ++n;
    S->arena_alloc.release(lv.a_off, lv.a_n);
    S->task_alloc.release(lv.t_off, lv.t_n);
    S->edge_alloc.release(lv.e_off, lv.e_n);
    lv.live = false;
    S->free_slots.push_back((int)slot);
    S->completed += 1;
    if (done && n >= cap) break;
  }
  *count = n;
  CtlLine stl;
  CK(cudaMemcpyAsync(&stl, &S->ctl->status, sizeof(CtlLine), cudaMemcpyDeviceToHost, S->cstream));
  CK(cudaStreamSynchronize(S->cstream));
  if (stl.v) return (int)stl.v;
  if (S->submitted > S->completed) return server_ensure_running(S);  // work owed: keep a kernel up
  return HQR_SUCCESS;
}

int hqr_server_counters(const hqr_server *S, uint32_t *out, int cap) {
  if (!S) return -1;
  if (!out || cap < 5) return -2;
  ServeCtl sc;
  CK(cudaMemcpy(&sc, S->sc, sizeof(ServeCtl), cudaMemcpyDeviceToHost));
  out[0] = sc.inbox_head.v;
  out[1] = sc.inbox_tail.v;
  out[2] = sc.stop.v;
  out[3] = sc.outstanding.v;
  out[4] = cudaStreamQuery(S->kstream) == cudaErrorNotReady ? 1u : 0u;
  return HQR_SUCCESS;
}

int hqr_server_progress(const hqr_server *S, int64_t ticket, int *done, int *total) {
  if (!S) return -1;
  if (!done || !total) return -3;
  for (size_t slot = 0; slot < S->live.size(); ++slot) {
    const hqr_server::Live &lv = S->live[slot];
    if (!lv.live || lv.seq != ticket) continue;
    CK(cudaMemcpy(done, S->req_done + slot, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(total, S->req_total + slot, sizeof(int), cudaMemcpyDeviceToHost));
    return HQR_SUCCESS;
  }
  return HQR_ERR_INTERNAL;
}

int hqr_server_stats(const hqr_server *S, int64_t *submitted, int64_t *completed, int *live, size_t *bytes_in_use) {
  if (!S) return -1;
  if (submitted) *submitted = S->submitted;
  if (completed) *completed = S->completed;
  if (live) *live = (int)(S->live.size() - S->free_slots.size());
  if (bytes_in_use) *bytes_in_use = S->arena_alloc.used() * 256;
  return HQR_SUCCESS;
}

int hqr_server_stop(hqr_server *S) {
  if (!S) return -1;
  if (!S->running) return HQR_SUCCESS;
  {
    const int rs = server_ensure_running(S);  // admitted work must finish before the kernel leaves
    if (rs) return rs;
  }
  const unsigned one = 1;
  CK(cudaMemcpyAsync(&S->sc->stop.v, &one, sizeof(unsigned), cudaMemcpyHostToDevice, S->cstream));
  CK(cudaStreamSynchronize(S->cstream));
  CK(cudaStreamSynchronize(S->kstream));
  S->running = false;
  CtlLine stl;
  CK(cudaMemcpy(&stl, &S->ctl->status, sizeof(CtlLine), cudaMemcpyDeviceToHost));
  const unsigned zero = 0;  // a later start serves again
  CK(cudaMemcpy(&S->sc->stop.v, &zero, sizeof(unsigned), cudaMemcpyHostToDevice));
  if (setup_done()) return HQR_ERR_CUDA;
  return (int)stl.v;
}

void hqr_server_free(hqr_server *S) {
  if (!S) return;
  if (S->running) hqr_server_stop(S);
  server_release(S);
  delete S;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free factorization (hqr_geqrf_r_noalloc).
//
// Some callers cannot allocate: code running where the device memory is
// owned by someone else's pool (a framework's caching allocator, a
// pre-reserved arena in a latency-critical service), where cudaMalloc would
// synchronize the device at the wrong moment, or where the process must not
// grow its heap after start-up. This entry point factors small problems
// using only the caller's buffers plus one fixed scratch array below, which
// is part of the library image: every GPU that loads the library holds it
// until the process exits. The task graph is built in static host storage,
// so the call does not allocate on the host either.
namespace {

constexpr size_t kNaScratchBytes = (size_t)16 << 20;  // 16 MiB device scratch
constexpr int kNaMaxM = 64, kNaMaxN = 16, kNaMaxTiles = 256;
constexpr int kNaMaxSlabs = 4;  // nb <= 64 with 16-column slabs
constexpr int kNaMaxTasks = 16384, kNaMaxEdges = 131072, kNaMaxReaders = 64;
constexpr int kNaMaxRes = kNaMaxTiles * (kNaMaxSlabs + 2);
constexpr int kNaMaxOps = 2 * kNaMaxTiles + kNaMaxN;
constexpr int kNaMaxDevices = 64;

// The device scratch. Host code must not pass `g_na_scratch` to a kernel
// (in host code it names a host-side stand-in); it uses the device address
// obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

struct NaHost {
  Task tasks[kNaMaxTasks];
  int indeg[kNaMaxTasks];
  int slots[kNumQueues * kShards * ((kNaMaxTasks + kShards - 1) / kShards)];
  int succ[kNaMaxEdges];
  int efrom[kNaMaxEdges], eto[kNaMaxEdges];
  int cnt[kNaMaxTasks + 1];
  int writer[kNaMaxRes];
  int nread[kNaMaxRes];
  int readers[kNaMaxRes][kNaMaxReaders];
  int deps[4 * kNaMaxReaders * (kNaMaxSlabs + 4)];
  long long pos[kNaMaxTiles];
  int state[kNaMaxM], tri[kNaMaxM];
  PanelOp ops[kNaMaxOps];
  Ctl ctl;
  Problem prob;
  int ntasks, nedges, ndeps, overflow;
  size_t pend_w[2 * kNaMaxSlabs + 8], pend_r[8];
  int npw, npr;
};
static NaHost g_na;
static void *g_na_dev_ptr[kNaMaxDevices];
static bool g_na_ready[kNaMaxDevices];

constexpr int kNaMaxDeps = (int)(sizeof(NaHost::deps) / sizeof(int));
constexpr int kNaMaxPendW = (int)(sizeof(NaHost::pend_w) / sizeof(size_t));
constexpr int kNaMaxPendR = (int)(sizeof(NaHost::pend_r) / sizeof(size_t));

void na_read(size_t res) {
  if (g_na.ndeps + 1 > kNaMaxDeps || g_na.npr >= kNaMaxPendR) {
    g_na.overflow = 1;
    return;
  }
  if (g_na.writer[res] >= 0) g_na.deps[g_na.ndeps++] = g_na.writer[res];
  g_na.pend_r[g_na.npr++] = res;
}
void na_write(size_t res) {
  if (g_na.ndeps + 1 + g_na.nread[res] > kNaMaxDeps || g_na.npw >= kNaMaxPendW) {
    g_na.overflow = 1;
    return;
  }
  if (g_na.writer[res] >= 0) g_na.deps[g_na.ndeps++] = g_na.writer[res];
  for (int q = 0; q < g_na.nread[res]; ++q) g_na.deps[g_na.ndeps++] = g_na.readers[res][q];
  g_na.pend_w[g_na.npw++] = res;
}
void na_add(const Task &t) {
  if (g_na.overflow) return;
  if (g_na.ntasks >= kNaMaxTasks) {
    g_na.overflow = 1;
    return;
  }
  const int id = g_na.ntasks++;
  std::sort(g_na.deps, g_na.deps + g_na.ndeps);
  const int nd = (int)(std::unique(g_na.deps, g_na.deps + g_na.ndeps) - g_na.deps);
  if (g_na.nedges + nd > kNaMaxEdges) {
    g_na.overflow = 1;
    return;
  }
  for (int q = 0; q < nd; ++q) {
    g_na.efrom[g_na.nedges] = g_na.deps[q];
    g_na.eto[g_na.nedges++] = id;
  }
  g_na.indeg[id] = nd;
  g_na.tasks[id] = t;
  for (int q = 0; q < g_na.npw; ++q) {
    g_na.writer[g_na.pend_w[q]] = id;
    g_na.nread[g_na.pend_w[q]] = 0;
  }
  for (int q = 0; q < g_na.npr; ++q) {
    const size_t res = g_na.pend_r[q];
    if (g_na.nread[res] >= kNaMaxReaders) {
      g_na.overflow = 1;
      return;
    }
    g_na.readers[res][g_na.nread[res]++] = id;
  }
  g_na.ndeps = g_na.npw = g_na.npr = 0;
}
Task na_task(int op, int prio, int i, int r, int k, int j, int c0, int cw) {
  Task t;
  t.op = (int8_t)op;
  t.prio = (int8_t)prio;
  t.trans = 1;
  t.tgt = 0;
  t.pid = 0;
  t.i = i;
  t.r = r;
  t.k = k;
  t.j = j;
  t.c0 = (int16_t)c0;
  t.cw = (int16_t)cw;
  t.blk = 0;
  t.pad_ = 0;
  t.succ_begin = t.succ_end = 0;
  return t;
}

// Validity rules of Sec. 2 (as hqr_validate_list), in static storage.
bool na_list_valid(int m, int n, const hqr_elim_t *list, size_t count) {
  const int K = std::min(m, n);
  for (int e = 0; e < m * K; ++e) g_na.pos[e] = -1;
  for (size_t q = 0; q < count; ++q) {
    const hqr_elim_t &r = list[q];
    if (r.k < 0 || r.k >= K || r.i <= r.k || r.i >= m || r.killer < r.k || r.killer >= m || r.killer == r.i)
      return false;
    if (r.kind != HQR_KIND_TS && r.kind != HQR_KIND_TT) return false;
    long long &p = g_na.pos[(size_t)r.k * m + r.i];
    if (p >= 0) return false;
    p = (long long)q;
  }
  for (int k = 0; k < K; ++k)
    for (int i = k + 1; i < m; ++i)
      if (g_na.pos[(size_t)k * m + i] < 0) return false;
  for (size_t q = 0; q < count; ++q) {
    const hqr_elim_t &r = list[q];
    for (int kp = 0; kp < r.k; ++kp) {
      if (r.i > kp && g_na.pos[(size_t)kp * m + r.i] > (long long)q) return false;
      if (r.killer > kp && g_na.pos[(size_t)kp * m + r.killer] > (long long)q) return false;
    }
    if (r.killer > r.k && g_na.pos[(size_t)r.k * m + r.killer] < (long long)q) return false;
  }
  for (int k = 0; k < K; ++k) {
    for (int i = 0; i < m; ++i) g_na.state[i] = 0;
    for (size_t q = 0; q < count; ++q) {
      const hqr_elim_t &r = list[q];
      if (r.k != k) continue;
      if (g_na.state[r.killer] == 2) return false;
      if (r.kind == HQR_KIND_TS && g_na.state[r.i] != 0) return false;
      g_na.state[r.killer] = 1;
      g_na.state[r.i] = 2;
    }
  }
  return true;
}

// The task graph of hqr_geqrf_r_noalloc for an m x n tile matrix and a
// valid list, built in the static host storage g_na: tasks with their
// successor ranges (succ_begin / succ_end into g_na.succ), in-degrees.
// Returns HQR_ERR_TOO_LARGE when a static table would overflow.
int na_build(int m, int n, int nb, int ib, const hqr_elim_t *list, size_t count) {
  (void)ib;
  const int w = std::min(16, nb);
  const int S = (nb + w - 1) / w;
  // operation sequence of Alg. 1 / Alg. 2 (as expand_ops)
  int nops = 0;
  for (int i = 0; i < m; ++i) g_na.tri[i] = -1;
  const int K = std::min(m, n);
  for (int k = 0; k < K; ++k) {
    bool any = false;
    for (size_t q = 0; q < count; ++q) {
      const hqr_elim_t &e = list[q];
      if (e.k != k) continue;
      any = true;
      if (g_na.tri[e.killer] != k) {
        g_na.ops[nops++] = {0, k, e.killer, e.killer};
        g_na.tri[e.killer] = k;
      }
      if (e.kind == HQR_KIND_TT && g_na.tri[e.i] != k) {
        g_na.ops[nops++] = {0, k, e.i, e.i};
        g_na.tri[e.i] = k;
      }
      g_na.ops[nops++] = {(int8_t)(e.kind == HQR_KIND_TS ? 1 : 2), k, e.i, e.killer};
    }
    if (!any) g_na.ops[nops++] = {0, k, k, k};
  }
  // task graph (same storage pieces and edges as build_factor_graph)
  const size_t per_tile = (size_t)S + 2;
  const size_t nres = (size_t)m * n * per_tile;
  for (size_t r = 0; r < nres; ++r) {
    g_na.writer[r] = -1;
    g_na.nread[r] = 0;
  }
  g_na.ntasks = g_na.nedges = g_na.ndeps = g_na.npw = g_na.npr = g_na.overflow = 0;
  auto slab = [&](int i, int j, int sl) { return ((size_t)j * m + i) * per_tile + (size_t)sl; };
  auto up = [&](int i, int j) { return ((size_t)j * m + i) * per_tile + (size_t)S; };
  auto lo = [&](int i, int j) { return ((size_t)j * m + i) * per_tile + (size_t)S + 1; };
  for (int q = 0; q < nops && !g_na.overflow; ++q) {
    const PanelOp &o = g_na.ops[q];
    const int k = o.k;
    const int pop = o.kind == 0 ? OP_GEQRT : (o.kind == 1 ? OP_TSQRT : OP_TTQRT);
    const int uop = o.kind == 0 ? OP_UNMQR : (o.kind == 1 ? OP_TSMQR : OP_TTMQR);
    if (o.kind == 0) {
      for (int sl = 0; sl < S; ++sl) na_write(slab(o.i, k, sl));
      na_write(up(o.i, k));
      na_write(lo(o.i, k));
    } else if (o.kind == 1) {
      na_write(up(o.r, k));
      for (int sl = 0; sl < S; ++sl) na_write(slab(o.i, k, sl));
      na_write(up(o.i, k));
      na_write(lo(o.i, k));
    } else {
      na_write(up(o.r, k));
      na_write(up(o.i, k));
    }
    na_add(na_task(pop, 0, o.i, o.kind == 0 ? o.i : o.r, k, k, 0, nb));
    for (int j = k + 1; j < n; ++j)
      for (int sl = 0; sl < S; ++sl) {
        if (o.kind == 0) {
          na_read(lo(o.i, k));
          na_write(slab(o.i, j, sl));
        } else {
          na_read(up(o.i, k));
          if (o.kind == 1) na_read(lo(o.i, k));
          na_write(slab(o.r, j, sl));
          na_write(slab(o.i, j, sl));
        }
        na_add(na_task(uop, j == k + 1 ? 1 : 2, o.i, o.kind == 0 ? o.i : o.r, k, j, sl * w,
                       std::min(w, nb - sl * w)));
      }
  }
  if (g_na.overflow) return HQR_ERR_TOO_LARGE;
  const int nt = g_na.ntasks;
  for (int t = 0; t <= nt; ++t) g_na.cnt[t] = 0;
  for (int e = 0; e < g_na.nedges; ++e) g_na.cnt[g_na.efrom[e] + 1]++;
  for (int t = 0; t < nt; ++t) g_na.cnt[t + 1] += g_na.cnt[t];
  for (int t = 0; t < nt; ++t) {
    g_na.tasks[t].succ_begin = g_na.cnt[t];
    g_na.tasks[t].succ_end = g_na.cnt[t + 1];
  }
  for (int e = 0; e < g_na.nedges; ++e) g_na.succ[g_na.cnt[g_na.efrom[e]]++] = g_na.eto[e];
  return HQR_SUCCESS;
}

// hqr_task_graph kind 6: the allocation-free entry point's graph (host only).
int na_task_graph(int m, int n, int nb, int ib, const hqr_elim_t *list, size_t count, int32_t *tasks,
                  int64_t task_cap, int64_t *succ_ptr, int32_t *succ, int64_t succ_cap, int64_t *ntasks,
                  int64_t *nedges) {
  if (nb > 64 || m > kNaMaxM || n > kNaMaxN || m * n > kNaMaxTiles) return HQR_ERR_TOO_LARGE;
  const int st = na_build(m, n, nb, ib, list, count);
  if (st) return st;
  *ntasks = g_na.ntasks;
  *nedges = g_na.nedges;
  if (!tasks) return HQR_SUCCESS;
  if (task_cap < *ntasks || !succ_ptr || (*nedges > 0 && (!succ || succ_cap < *nedges))) return HQR_ERR_CAPACITY;
  for (int q = 0; q < g_na.ntasks; ++q) {
    const Task &t = g_na.tasks[q];
    const int32_t row[10] = {t.op, t.blk, t.i, t.r, t.k, t.j, t.c0, t.cw, t.trans, t.tgt};
    std::memcpy(tasks + 10 * (size_t)q, row, sizeof(row));
    succ_ptr[q] = t.succ_begin;
  }
  succ_ptr[g_na.ntasks] = g_na.nedges;
  if (g_na.nedges) std::memcpy(succ, g_na.succ, sizeof(int32_t) * (size_t)g_na.nedges);
  return HQR_SUCCESS;
}

size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int hqr_geqrf_r_noalloc(const void *dA, int M, int N, int lda, int nb, int ib,
                                   const hqr_elim_t *list, size_t count, void *dR, int ldr, void *stream) {
  if (!dA) return -1;
  if (M < 1) return -2;
  if (N < 1 || N > M) return -3;
  if (lda < M) return -4;
  if (nb < 8 || nb % 8) return -5;
  if (ib < 2 || ib % 2 || nb % ib || (ib > 16 && ib != 32)) return -6;
  if (!list) return -7;
  if (!dR) return -9;
  if (ldr < N) return -10;
  if (nb > 64) return HQR_ERR_TOO_LARGE;
  const int m = (M + nb - 1) / nb, n = (N + nb - 1) / nb;
  if (m > kNaMaxM || n > kNaMaxN || m * n > kNaMaxTiles) return HQR_ERR_TOO_LARGE;
  if (!na_list_valid(m, n, list, count)) return -7;
  cudaStream_t s = (cudaStream_t)stream;
  {  // the call stages from host memory and synchronizes the stream: it cannot be captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return -11;
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HQR_ERR_CUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return HQR_ERR_TOO_LARGE;
  if (!g_na_ready[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return HQR_ERR_CUDA;
    g_na_dev_ptr[dev] = p;
    g_na_ready[dev] = true;
  }
  const int w = std::min(16, nb), wt = std::min(16, nb), vc = std::min(ib, 16);
  {
    const int bst = na_build(m, n, nb, ib, list, count);
    if (bst) return bst;
  }
  const int nt = g_na.ntasks;
  for (size_t q = 0; q < slot_count(nt); ++q) g_na.slots[q] = 0;
  init_ready(g_na.tasks, g_na.indeg, nt, g_na.slots, g_na.ctl);
  // scratch layout
  const size_t a_bytes = na_align(sizeof(double) * (size_t)m * nb * n * nb);
  const size_t t_bytes = na_align(sizeof(double) * (size_t)m * n * 2 * ib * nb);
  const size_t k_bytes = na_align(sizeof(Task) * nt);
  const size_t s_bytes = na_align(sizeof(int) * std::max(g_na.nedges, 1));
  const size_t d_bytes = na_align(sizeof(int) * nt);
  const size_t q_bytes = na_align(sizeof(int) * slot_count(nt));
  const size_t c_bytes = na_align(sizeof(Ctl));
  const size_t p_bytes = na_align(sizeof(Problem));
  if (a_bytes + t_bytes + k_bytes + s_bytes + d_bytes + q_bytes + c_bytes + p_bytes > kNaScratchBytes)
    return HQR_ERR_TOO_LARGE;
  unsigned char *base = (unsigned char *)g_na_dev_ptr[dev];
  double *dws = (double *)base;
  double *dT = (double *)(base + a_bytes);
  Task *dtasks = (Task *)(base + a_bytes + t_bytes);
  int *dsucc = (int *)(base + a_bytes + t_bytes + k_bytes);
  int *dindeg = (int *)(base + a_bytes + t_bytes + k_bytes + s_bytes);
  int *dslots = (int *)(base + a_bytes + t_bytes + k_bytes + s_bytes + d_bytes);
  Ctl *dctl = (Ctl *)(base + a_bytes + t_bytes + k_bytes + s_bytes + d_bytes + q_bytes);
  Problem *dprob = (Problem *)(base + a_bytes + t_bytes + k_bytes + s_bytes + d_bytes + q_bytes + c_bytes);
  g_na.prob.A = dws;
  g_na.prob.T = dT;
  g_na.prob.B = nullptr;
  g_na.prob.m = m;
  g_na.prob.n = n;
  g_na.prob.nb = nb;
  g_na.prob.ib = ib;
  g_na.prob.w = w;
  g_na.prob.wt = wt;
  g_na.prob.vc = vc;
  g_na.prob.wb = w;
  if (cudaMemcpyAsync(dtasks, g_na.tasks, sizeof(Task) * nt, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (g_na.nedges > 0 &&
       cudaMemcpyAsync(dsucc, g_na.succ, sizeof(int) * g_na.nedges, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemcpyAsync(dindeg, g_na.indeg, sizeof(int) * nt, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dslots, g_na.slots, sizeof(int) * slot_count(nt), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(dctl, &g_na.ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dprob, &g_na.prob, sizeof(Problem), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return HQR_ERR_CUDA;
  const long long total = (long long)m * nb * n * nb;
  pack_tiles<double><<<grid_for(total), 256, 0, s>>>((const double *)dA, lda, M, N, (double *)dws, m, nb, total);
  EngineParams p{};
  p.probs = dprob;
  p.trace = nullptr;
  p.tasks = dtasks;
  p.ntasks = nt;
  p.succ = dsucc;
  p.indeg = dindeg;
  p.slots = dslots;
  p.ctl = dctl;
  p.timeout_ns = g_timeout_ns;
  const size_t smem = engine_smem_bytes<double>(nb, ib, w, wt, vc);
  int sms = 0, per_sm = 0;
  if (cudaFuncSetAttribute(hqr_sched<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hqr_sched<double, false>, NT, smem) != cudaSuccess ||
      per_sm < 1)
    return HQR_ERR_CUDA;
  hqr_sched<double, false><<<std::max(1, std::min(sms * per_sm, nt)), NT, smem, s>>>(p);
  unpack_tiles<double><<<grid_for((long long)N * N), 256, 0, s>>>((const double *)dws, m, nb, (double *)dR, ldr, N,
                                                                 N, 1);
  if (cudaGetLastError() != cudaSuccess) return HQR_ERR_CUDA;
  if (cudaMemcpyAsync(&g_na.ctl.status, &dctl->status, sizeof(CtlLine), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HQR_ERR_CUDA;
  return (int)g_na.ctl.status.v;
}
