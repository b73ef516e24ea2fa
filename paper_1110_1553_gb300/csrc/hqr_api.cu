// C ABI of the library (include/hqr.h): argument checks, workspace and task
// graph management, and the launches of the device engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/hqr.h"
#include "engine_fp64.cuh"
#include "hqr_internal.h"

using namespace hqr;

namespace {

thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;
int64_t g_timeout_ns = 20000000000ll;

bool cuda_ok(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}
#define CK(call)                                  \
  do {                                            \
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

int upload_graph(const Graph &g, DevGraph &d) {
  const int nt = (int)g.tasks.size();
  d.ntasks = nt;
  d.nedges = g.nedges;
  std::vector<int> slots((size_t)kNumQueues * nt, 0);
  Ctl ctl;
  std::memset(&ctl, 0, sizeof(ctl));
  for (int t = 0; t < nt; ++t)
    if (g.indeg[t] == 0) {
      const int q = g.tasks[t].prio;
      slots[(size_t)q * nt + ctl.tail[q]++] = t + 1;
    }
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
  return HQR_SUCCESS;
}

// Tile-major packing of a column-major matrix, zero padded to whole tiles.
__global__ void pack_tiles(const double *__restrict__ A, long long lda, int M, int N, double *__restrict__ ws,
                           int m, int nb, long long total) {
  const long long nb2 = (long long)nb * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long tile = e / nb2;
    const int w = (int)(e - tile * nb2);
    const int cc = w / nb, rr = w - cc * nb;
    const int ti = (int)(tile % m), tj = (int)(tile / m);
    const int row = ti * nb + rr, col = tj * nb + cc;
    ws[e] = (row < M && col < N) ? A[(long long)col * lda + row] : 0.0;
  }
}

// Inverse of pack_tiles for the padded Mp x Np matrix; `upper_only` keeps
// rows <= col and zeroes the rest (R), limited to rows, cols < lim.
__global__ void unpack_tiles(const double *__restrict__ ws, int m, int nb, double *__restrict__ out,
                             long long ld, int rows, int cols, int upper_only) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(e / rows), row = (int)(e - (long long)col * rows);
    const int ti = row / nb, tj = col / nb;
    double v = ws[((size_t)tj * m + ti) * nb * nb + (size_t)(col - tj * nb) * nb + (row - ti * nb)];
    if (upper_only && row > col) v = 0.0;
    out[(long long)col * ld + row] = v;
  }
}

// Right-hand side (M x nrhs) into blocks of nb rows x wa columns: block
// (r, s) at ((s*m + r)*nb*wa), column-major inside.
__global__ void pack_rhs(const double *__restrict__ B, long long ldb, int M, int nrhs, double *__restrict__ Bw,
                         int m, int nb, int wa, long long total) {
  const long long bs = (long long)nb * wa;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / bs;
    const int w = (int)(e - blk * bs);
    const int cc = w / nb, rr = w - cc * nb;
    const int r = (int)(blk % m), s = (int)(blk / m);
    const int row = r * nb + rr, col = s * wa + cc;
    Bw[e] = (row < M && col < nrhs) ? B[(long long)col * ldb + row] : 0.0;
  }
}

__global__ void unpack_rhs(const double *__restrict__ Bw, double *__restrict__ B, long long ldb, int M, int nrhs,
                           int m, int nb, int wa) {
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
__global__ void trsv_diag(const double *__restrict__ ws, int m, int nb, int i, int nbi, double *X, long long ldx,
                          int *singular) {
  __shared__ double xs[256];
  double *x = X + (long long)blockIdx.x * ldx + (long long)i * nb;
  const double *Rt = ws + ((size_t)i * m + i) * nb * nb;
  for (int r = threadIdx.x; r < nbi; r += blockDim.x) xs[r] = x[r];
  __syncthreads();
  for (int r = nbi - 1; r >= 0; --r) {
    if (threadIdx.x == 0) {
      const double d = Rt[(size_t)r * nb + r];
      if (d == 0.0) {
        atomicExch(singular, 1);
        xs[r] = 0.0;
      } else {
        xs[r] = xs[r] / d;
      }
    }
    __syncthreads();
    const double xr = xs[r];
    for (int l = threadIdx.x; l < r; l += blockDim.x) xs[l] = fma(-Rt[(size_t)r * nb + l], xr, xs[l]);
    __syncthreads();
  }
  for (int r = threadIdx.x; r < nbi; r += blockDim.x) x[r] = xs[r];
}

// c[0 : i*nb) -= R[0 : i*nb, columns of tile i] x_i.
__global__ void trsv_update(const double *__restrict__ ws, int m, int nb, int i, int nbi, double *X,
                            long long ldx) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= i * nb) return;
  const int ti = row / nb, rr = row - ti * nb;
  const double *Rt = ws + ((size_t)i * m + ti) * nb * nb;
  const double *x = X + (long long)blockIdx.y * ldx + (long long)i * nb;
  double s = 0.0;
  for (int c = 0; c < nbi; ++c) s = fma(Rt[(size_t)c * nb + rr], x[c], s);
  X[(long long)blockIdx.y * ldx + row] -= s;
}

int grid_for(int n) { return std::max(1, std::min(4096, (n + 255) / 256)); }

}  // namespace

struct hqr_factors {
  int M = 0, N = 0, Mp = 0, Np = 0, m = 0, n = 0, nb = 0, ib = 0, prec = 0;
  int w = 0, wt = 0, vc = 0, wa = 0;
  size_t smem = 0;
  int grid = 0;
  std::vector<hqr_elim_t> list;
  std::vector<PanelOp> ops;
  double *dA = nullptr, *dT = nullptr, *dBw = nullptr;
  size_t bw_cap = 0;
  DevGraph fg;
  std::map<std::pair<int, int>, DevGraph> ag;  // (trans, nslab) -> apply graph
  Ctl *last_ctl = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  int64_t debug_task = -1;
  int debug_base = -1;
};

namespace {

int ctas_for(const hqr_factors *F, size_t smem, int ntasks, int *grid) {
  static bool attr_set = false;
  static size_t attr_smem = 0;
  if (!attr_set || attr_smem < smem) {
    CK(cudaFuncSetAttribute(hqr_sched_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
    attr_smem = smem;
  }
  int dev = 0, sms = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hqr_sched_fp64, NT, smem));
  if (per_sm < 1) {
    g_last_error = "scheduler kernel does not fit on an SM";
    return HQR_ERR_CUDA;
  }
  (void)F;
  *grid = std::max(1, std::min(sms * per_sm, ntasks));
  return HQR_SUCCESS;
}

int run_graph(hqr_factors *F, DevGraph &g, double *C, long long cstride, int w, cudaStream_t s) {
  EngineParams p;
  p.A = F->dA;
  p.T = F->dT;
  p.C = C;
  p.cstride = cstride;
  p.m = F->m;
  p.n = F->n;
  p.nb = F->nb;
  p.ib = F->ib;
  p.w = w;
  p.wt = F->wt;
  p.vc = F->vc;
  p.lds = F->nb + 2;
  p.tasks = g.tasks;
  p.ntasks = g.ntasks;
  p.succ = g.succ;
  p.indeg = g.indeg;
  p.slots = g.slots;
  p.ctl = g.ctl;
  p.timeout_ns = g_timeout_ns;
  const size_t smem = engine_smem_bytes(F->nb, F->ib, w, F->wt, F->vc);
  int grid = 0;
  int st = ctas_for(F, smem, g.ntasks, &grid);
  if (st) return st;
  CK(cudaMemcpyAsync(g.indeg, g.indeg0, sizeof(int) * g.ntasks, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(g.slots, g.slots0, sizeof(int) * (size_t)kNumQueues * g.ntasks,
                     cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(g.ctl, g.ctl0, sizeof(Ctl), cudaMemcpyDeviceToDevice, s));
  if (!F->ev0) {
    CK(cudaEventCreate(&F->ev0));
    CK(cudaEventCreate(&F->ev1));
  }
  CK(cudaEventRecord(F->ev0, s));
  hqr_sched_fp64<<<grid, NT, smem, s>>>(p);
  CK(cudaGetLastError());
  CK(cudaEventRecord(F->ev1, s));
  F->timed = true;
  g_launches += 1;
  F->last_ctl = g.ctl;
  F->grid = grid;
  return HQR_SUCCESS;
}

int read_status(hqr_factors *F, cudaStream_t s) {
  CK(cudaStreamSynchronize(s));
  if (!F->last_ctl) return HQR_SUCCESS;
  Ctl c;
  CK(cudaMemcpy(&c, F->last_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  if (c.status != 0) return c.status;
  return HQR_SUCCESS;
}

int pack_a(hqr_factors *F, const double *dA, int lda, cudaStream_t s) {
  const long long total = (long long)F->Mp * F->Np;
  pack_tiles<<<grid_for((int)std::min<long long>(total, 1 << 30)), 256, 0, s>>>(dA, lda, F->M, F->N, F->dA,
                                                                                 F->m, F->nb, total);
  CK(cudaGetLastError());
  g_launches += 1;
  return HQR_SUCCESS;
}

}  // namespace

extern "C" {

void hqr_set_timeout_ms(int64_t ms) { g_timeout_ns = (ms > 0 ? ms : 1) * 1000000ll; }

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
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

int hqr_geqrf(const void *dA, int M, int N, int lda, int prec, int nb, int ib, const hqr_elim_t *list,
              size_t count, hqr_factors **out, void *stream) {
  g_launches = 0;
  if (!dA) return -1;
  if (M < 1) return -2;
  if (N < 1 || N > M) return -3;
  if (lda < M) return -4;
  if (prec != HQR_FP64) return -5;
  if (nb < 8 || nb > 256 || nb % 8) return -6;
  if (ib < 2 || ib % 2 || nb % ib || (ib > 16 && ib != 32)) return -7;
  if (!out) return -10;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
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
  F->w = std::min(16, nb);
  F->wt = nb > 128 ? 8 : std::min(16, nb);
  F->vc = nb > 128 ? std::min(ib, 8) : std::min(ib, 16);
  F->wa = std::min(16, nb);
  // elimination list
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
    int st = hqr_elim_list(F->m, F->n, 4, 1, HQR_GREEDY, HQR_GREEDY, F->list.data(), cnt, &cnt);
    if (st) {
      delete F;
      return HQR_ERR_INTERNAL;
    }
  }
  F->ops = expand_ops(F->list.data(), F->list.size(), F->m, F->n);
  Graph g = build_factor_graph(F->ops, F->m, F->n, nb, F->w);
  int st = upload_graph(g, F->fg);
  if (!st) {
    const size_t tsz = (size_t)F->m * F->n * 2 * ib * nb;
    if (!cuda_ok(cudaMalloc(&F->dA, sizeof(double) * (size_t)F->Mp * F->Np), "cudaMalloc(A)") ||
        !cuda_ok(cudaMalloc(&F->dT, sizeof(double) * tsz), "cudaMalloc(T)") ||
        !cuda_ok(cudaMemsetAsync(F->dT, 0, sizeof(double) * tsz, s), "memset(T)"))
      st = HQR_ERR_NOMEM;
  }
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
  int st = pack_a(F, (const double *)dA, lda, s);
  if (st) return st;
  return run_graph(F, F->fg, F->dA, (long long)F->nb * F->nb, F->w, s);
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
  unpack_tiles<<<grid_for(F->N * F->N), 256, 0, s>>>(F->dA, F->m, F->nb, (double *)dR, ldr, F->N, F->N, 1);
  CK(cudaGetLastError());
  return HQR_SUCCESS;
}

int hqr_get_tiles(const hqr_factors *F, void *dOut, int ld, void *stream) {
  if (!F) return -1;
  if (!dOut) return -2;
  if (ld < F->Mp) return -3;
  cudaStream_t s = (cudaStream_t)stream;
  unpack_tiles<<<grid_for(F->Mp * F->Np), 256, 0, s>>>(F->dA, F->m, F->nb, (double *)dOut, ld, F->Mp, F->Np,
                                                       0);
  CK(cudaGetLastError());
  return HQR_SUCCESS;
}

int hqr_get_t(const hqr_factors *F, void *dT, void *stream) {
  if (!F) return -1;
  if (!dT) return -2;
  const size_t tsz = (size_t)F->m * F->n * 2 * F->ib * F->nb;
  CK(cudaMemcpyAsync(dT, F->dT, sizeof(double) * tsz, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
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
  const int wa = F->wa;
  const int nslab = (nrhs + wa - 1) / wa;
  const size_t need = (size_t)F->Mp * nslab * wa;
  if (need > F->bw_cap) {
    cudaFree(F->dBw);
    F->dBw = nullptr;
    F->bw_cap = 0;
    if (!cuda_ok(cudaMalloc(&F->dBw, sizeof(double) * need), "cudaMalloc(B)")) return HQR_ERR_NOMEM;
    F->bw_cap = need;
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
  pack_rhs<<<grid_for((int)std::min<long long>(total, 1 << 30)), 256, 0, s>>>(
      (const double *)dB, ldb, F->M, nrhs, F->dBw, F->m, F->nb, wa, total);
  CK(cudaGetLastError());
  g_launches += 1;
  int st = run_graph(F, it->second, F->dBw, (long long)F->nb * wa, wa, s);
  if (st) return st;
  unpack_rhs<<<grid_for((int)std::min<long long>((long long)F->M * nrhs, 1 << 30)), 256, 0, s>>>(
      F->dBw, (double *)dB, ldb, F->M, nrhs, F->m, F->nb, wa);
  CK(cudaGetLastError());
  g_launches += 1;
  return read_status(F, s);
}

int hqr_gels(const void *dA, int M, int N, int lda, const void *db, int ldb, int nrhs, void *dx, int ldx,
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
  double *c = nullptr;
  int *dsing = nullptr;
  int64_t launches = g_launches;
  do {
    if (!cuda_ok(cudaMalloc(&c, sizeof(double) * (size_t)M * nrhs), "cudaMalloc(c)") ||
        !cuda_ok(cudaMalloc(&dsing, sizeof(int)), "cudaMalloc(flag)")) {
      st = HQR_ERR_NOMEM;
      break;
    }
    if (!cuda_ok(cudaMemcpy2DAsync(c, sizeof(double) * M, db, sizeof(double) * ldb, sizeof(double) * M, nrhs,
                                   cudaMemcpyDeviceToDevice, s),
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
      trsv_diag<<<nrhs, 256, 0, s>>>(F->dA, F->m, F->nb, i, nbi, c, M, dsing);
      launches += 1;
      if (i > 0) {
        dim3 gr((i * F->nb + 255) / 256, nrhs);
        trsv_update<<<gr, 256, 0, s>>>(F->dA, F->m, F->nb, i, nbi, c, M);
        launches += 1;
      }
    }
    if (!cuda_ok(cudaGetLastError(), "trsv") ||
        !cuda_ok(cudaMemcpy2DAsync(dx, sizeof(double) * ldx, c, sizeof(double) * M, sizeof(double) * N, nrhs,
                                   cudaMemcpyDeviceToDevice, s),
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
  int base = 0;
  // the pristine in-degree lives on the device; keep the original on the host
  if (F->debug_task != task || F->debug_base < 0) {
    CK(cudaMemcpy(&base, F->fg.indeg0 + task, sizeof(int), cudaMemcpyDeviceToHost));
    if (F->debug_task >= 0 && F->debug_task != task) return HQR_ERR_INTERNAL;
    F->debug_task = task;
    F->debug_base = base;
  }
  const int v = F->debug_base + extra;
  CK(cudaMemcpy(F->fg.indeg0 + task, &v, sizeof(int), cudaMemcpyHostToDevice));
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
  if (F->ev0) cudaEventDestroy(F->ev0);
  if (F->ev1) cudaEventDestroy(F->ev1);
  delete F;
}

}  // extern "C"
