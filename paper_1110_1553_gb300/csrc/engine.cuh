// Tile kernels of tile Householder QR and the persistent task scheduler that
// runs them (sm_103a), for FP64 and FP32 storage and arithmetic.
//
// Every task of the graph (GEQRT, TSQRT, TTQRT and the UNMQR, TSMQR, TTMQR
// updates of Alg. 2) is executed by one CTA of a persistent kernel. A CTA
// takes the highest-priority ready task from device queues, stages its tile
// data in shared memory with bulk copies (the TMA engine; one copy per tile
// column, completion counted on an mbarrier), computes, writes the tiles back
// and releases its successors: each successor whose count of missing inputs
// drops to zero is pushed to a queue (Sec. 4.2, "Execution scheme": each
// kernel fires as soon as its dependencies are satisfied). Tasks of several
// independent problems can share one graph and one launch (each task names
// its problem).
//
// Arithmetic (compact-WY Householder, reflectors grouped ib at a time):
//   column j of (alpha, x2): s = ||x2|| (sum of squares; a max-scaled second
//   pass when the sum under- or overflows), beta = -sign(alpha) hypot(alpha,
//   s) with sign(+-0) = +1, tau = (beta - alpha) / beta, v = (1, x2/(alpha -
//   beta)); s == 0 gives the identity (tau = 0, beta = alpha).
//   T of a block: T[j,j] = tau_j, T[:j,j] = -tau_j T[:j,:j] (V[:,:j]^T v_j).
//   Q^T C = C - V T^T V^T C (blocks in ascending order); Q C uses T and the
//   descending order.
// Norm reductions use warp shuffles and a per-warp shared-memory stage.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "hqr_internal.h"
#include "ptx.cuh"
#include "tc.cuh"

namespace hqr {

constexpr int NT = 256;         // threads per CTA
constexpr int NWARP = NT / 32;  // warps per CTA
constexpr int IBMAX = 32;       // largest inner block

template <typename Real>
struct RealTraits;
template <>
struct RealTraits<double> {
  static constexpr double tiny = 1e-280, huge = 1e280;  // sum-of-squares range kept unscaled
};
template <>
struct RealTraits<float> {
  static constexpr float tiny = 1e-30f, huge = 1e30f;
};
// shared-memory column padding (elements): keeps every staged column on a
// 16-byte boundary and spreads columns over banks
template <typename Real>
__host__ __device__ constexpr int smem_pad() { return 16 / (int)sizeof(Real); }

// Ready queues are sharded: a task goes to shard (task id mod kShards) of its
// priority class, so each shard holds at most ceil(ntasks / kShards) tasks.
// CTAs look at their home shard first. Every counter sits on its own 128-byte
// line so that the atomics of different shards do not contend.
constexpr int kShards = 8;
struct alignas(128) CtlLine {
  unsigned v;
  int aux;
  unsigned pad[30];
};

// Device control words of one graph run.
struct Ctl {
  CtlLine head[kNumQueues * kShards];
  CtlLine tail[kNumQueues * kShards];
  CtlLine done;
  CtlLine status;  // v: status code, aux: task that failed (or -1)
};

__host__ __device__ inline int shard_cap(int ntasks) { return (ntasks + kShards - 1) / kShards; }

// Initial ready slots and control words for a graph (host side): every task
// with no inputs is placed in its queue shard.
inline void init_ready(const Task *tasks, const int *indeg, int ntasks, int *slots, Ctl &ctl) {
  std::memset(&ctl, 0, sizeof(Ctl));
  const int cap = shard_cap(ntasks);
  for (int t = 0; t < ntasks; ++t)
    if (indeg[t] == 0) {
      const int qs = tasks[t].prio * kShards + t % kShards;
      slots[(size_t)qs * cap + ctl.tail[qs].v++] = t + 1;
    }
}
inline size_t slot_count(int ntasks) { return (size_t)kNumQueues * kShards * shard_cap(ntasks); }

// One problem of a (possibly batched) task graph.
struct alignas(16) Problem {
  void *A;            // tile workspace: tile (i, j) at ((j*m + i)*nb*nb), column-major
  void *T;            // T factors: record ((k*m + i)*2 + which) of tstr elements, ib x nb column-major first
  void *B;            // right-hand-side blocks: block (r, s) at ((s*m + r)*nb*wb)
  int m, n, nb, ib;
  int w;              // width of an update task's column slab (max)
  int wt;             // slab width of the trailing update inside panel tasks
  int vc;             // V columns staged per chunk in update tasks (divides ib)
  int wb;             // right-hand-side block width
  // least-squares solves (FP64 vectors; unused by plain factorizations)
  int M, N;           // true sizes (the tile workspace is zero padded)
  const void *A0;     // the caller's matrix, column-major, storage precision
  long long lda0;
  const double *b;    // right-hand side (M)
  double *x, *r, *g;  // solution (N), residual (m*nb), work vector (n*nb)
  double *gp;         // partial sums of A^T r: (row chunk, column) pairs (sum, compensation)
  double *rp;         // partial sums of A x: (column chunk, row) pairs (sum, compensation)
  double *rinv;       // inverses of the diagonal R tiles, n tiles of nb x nb, column-major
  int *status;        // per-problem status word (HQR_ERR_SINGULAR)
  int tc;             // FP32 tiles of 128 on the tensor-core kernels (ib = nb: one full T per tile)
  int tstr;           // elements per T record (ib * nb; tensor-core problems: split images [+ T])
  int t32;            // tensor-core problems: the records keep the FP32 T (apply Q, read T)
  int maxit;          // tolerance-stopped refinement: rounds at most (0: fixed rounds)
  double tol;         // tolerance-stopped refinement: stop when ||d||_2 / ||x||_2 <= tol
  RefineState *rs;    // tolerance-stopped refinement state (nullptr otherwise)
  double *rn;         // tolerance-stopped refinement: per tile of x, sum d^2 and sum x^2 of a round
  long long pad2_;
};
static_assert(sizeof(Problem) % 16 == 0, "Problem is read in 16-byte pieces");

struct EngineParams {
  const Problem *probs;
  const Task *tasks;
  int ntasks;
  const int *succ;
  int *indeg;
  int *slots;          // kNumQueues x kShards x shard_cap(ntasks) slots (task id + 1, 0 = empty)
  Ctl *ctl;
  long long timeout_ns;
  unsigned long long *trace;  // optional: per task start, end (globaltimer), SM id
  int tc;                     // some problem uses the tensor-core kernels (launch the TC variant)
};

template <typename Real>
struct Shared {
  uint64_t bar;
  int task;
  int abort;
  int vskip, vcomp;  // vector tasks of tolerance-stopped rounds: skip the task, compensated sums
  int norelease;     // the task released none of its successors (a gate that cancelled its rounds)
  int kept;          // a successor the last task made ready and this CTA runs next (-1: none)
  int popped;        // the task warp 1 claimed (-1: none, or finished)
  Real red[2 * NWARP];
  Real tau[IBMAX];
  Real wv[IBMAX];
  Real bc[4];
};

// ---------------------------------------------------------------- helpers --

// Geometry of one task's problem, read once per task from global memory.
template <typename Real>
struct Geo {
  Real *A, *T, *B;
  int m, n, nb, ib, w, wt, vc, wb, lds, ldt, t32;
  size_t tstr;
  __device__ explicit Geo(const Problem &P)
      : A((Real *)P.A), T((Real *)P.T), B((Real *)P.B), m(P.m), n(P.n), nb(P.nb), ib(P.ib), w(P.w),
        wt(P.wt), vc(P.vc), wb(P.wb), lds(P.nb + smem_pad<Real>()), ldt(P.ib + smem_pad<Real>()), t32(P.t32),
        tstr(P.tstr > 0 ? (size_t)P.tstr : (size_t)P.ib * P.nb) {}
  __device__ Real *tile(int i, int j) const { return A + ((size_t)j * m + i) * (size_t)nb * nb; }
  __device__ Real *tfac(int which, int i, int k) const { return T + (((size_t)k * m + i) * 2 + which) * tstr; }
  // columns [t.c0, t.c0 + t.cw) of the target block of row `row`
  __device__ Real *target(const Task &t, int row) const {
    if (t.tgt == 0) return A + ((size_t)t.j * m + row) * (size_t)nb * nb + (size_t)t.c0 * nb;
    return B + ((size_t)t.j * m + row) * (size_t)nb * wb + (size_t)t.c0 * nb;
  }
};

__device__ __forceinline__ void set_error(const EngineParams &p, int code, int task) {
  if (atomicCAS((int *)&p.ctl->status.v, 0, code) == 0) p.ctl->status.aux = task;
}

template <typename Real>
struct Copy {
  Real *dst;
  int ldd;
  const Real *src;
  long long lds;
  int nrows, ncols;
};

// Stage up to 3 column-blocks global -> shared with bulk copies, one copy per
// column, and wait for them (bounded). Callers sync before (dst free).
template <typename Real>
__device__ void stage(const EngineParams &p, Shared<Real> &sh, const Copy<Real> *cp, int ncp,
                      uint32_t &phase) {
  uint32_t total = 0;
  for (int q = 0; q < ncp; ++q)
    if (cp[q].nrows > 0 && cp[q].ncols > 0)
      total += (uint32_t)cp[q].nrows * (uint32_t)sizeof(Real) * (uint32_t)cp[q].ncols;
  if (total == 0) return;
  if (threadIdx.x < 32) {
    ptx::fence_proxy_async();
    if (threadIdx.x == 0) ptx::mbar_arrive_expect_tx(&sh.bar, total);
    __syncwarp();
    for (int q = 0; q < ncp; ++q) {
      if (cp[q].nrows <= 0) continue;
      const uint32_t bytes = (uint32_t)cp[q].nrows * (uint32_t)sizeof(Real);
      for (int c = threadIdx.x; c < cp[q].ncols; c += 32)
        ptx::bulk_g2s(cp[q].dst + (size_t)c * cp[q].ldd, cp[q].src + (long long)c * cp[q].lds, bytes,
                      &sh.bar);
    }
  }
  if (!ptx::mbar_try_wait(&sh.bar, phase)) {
    const uint64_t t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(&sh.bar, phase)) {
      if (sh.abort || ptx::globaltimer() - t0 > (uint64_t)p.timeout_ns) {
        sh.abort = 1;
        break;
      }
    }
  }
  phase ^= 1u;
  __syncthreads();
  if (sh.abort && threadIdx.x == 0) set_error(p, HQR_ERR_TIMEOUT, -1);
}

// Write an nrows x ncols block from shared to global (coalesced along rows).
// mode 0: all; 1: only rows <= roff + col (upper part incl. diagonal).
template <typename Real>
__device__ void store_cols(Real *g, long long ldg, const Real *s, int ldsm, int nrows, int ncols, int mode,
                           int roff) {
  const int total = nrows * ncols;
  for (int e = threadIdx.x; e < total; e += NT) {
    const int c = e / nrows, r = e - c * nrows;
    if (mode == 1 && r > roff + c) continue;
    g[(long long)c * ldg + r] = s[(size_t)c * ldsm + r];
  }
}

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; every thread gets the same value (fixed order). Only
// threads below `nact` hold nonzero values, so warps beyond them skip their
// reduction, and one thread adds the warps' partial sums and broadcasts the
// total: in FP64 a warp-wide add occupies the SM's FP64 pipe for 16 cycles
// whether or not its lanes need the result.
template <typename Real>
__device__ Real block_sum(Real v, Shared<Real> &sh, int nact = NT) {
  if ((int)(threadIdx.x & ~31u) < nact) v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    Real t = 0;
#pragma unroll
    for (int q = 0; q < NWARP; ++q) t += sh.red[q];
    sh.red[NWARP] = t;
  }
  __syncthreads();
  return sh.red[NWARP];
}

template <typename Real>
__device__ Real block_max(Real v, Shared<Real> &sh, int nact = NT) {
  if ((int)(threadIdx.x & ~31u) < nact)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    Real t = 0;
#pragma unroll
    for (int q = 0; q < NWARP; ++q) t = fmax(t, sh.red[q]);
    sh.red[NWARP] = t;
  }
  __syncthreads();
  return sh.red[NWARP];
}

// FP32 versions of the two GEMM phases with register blocking and 16-byte
// shared-memory loads: each thread owns a 4 x 4 (W = V^T C) or 4 x 8
// (C -= V W) block of outputs, so an FFMA costs at most one eighth of a
// shared-memory access instead of two. K must be a multiple of 4 (true for
// FP32 tiles: nb, ib and every row offset are multiples of 4).
__device__ void gemm_tn_f32(float *W, int ldw, const float *V, int ldv, const float *Cm, int ldc, int K, int Mi,
                            int Nj, const float *Cinit, int ldi, float *scr) {
  const int ti = (Mi + 3) >> 2, tj = (Nj + 3) >> 2, T = ti * tj;
  int G = NT / T;
  if (G < 1) G = 1;
  if (G > 4) G = 4;
  int Kc = (K + G - 1) / G;
  Kc = (Kc + 3) & ~3;
  for (int u = threadIdx.x; u < T * G; u += NT) {
    const int mt = u % T, g = u / T;
    const int i0 = (mt % ti) * 4, j0 = (mt / ti) * 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const int k0 = g * Kc, k1 = min(K, k0 + Kc);
    const float *vp[4], *cp[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) vp[a] = V + (size_t)min(i0 + a, Mi - 1) * ldv;
#pragma unroll
    for (int b = 0; b < 4; ++b) cp[b] = Cm + (size_t)min(j0 + b, Nj - 1) * ldc;
    for (int k = k0; k < k1; k += 4) {
      float4 v4[4], c4[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) v4[a] = *reinterpret_cast<const float4 *>(vp[a] + k);
#pragma unroll
      for (int b = 0; b < 4; ++b) c4[b] = *reinterpret_cast<const float4 *>(cp[b] + k);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b] = fmaf(v4[a].x, c4[b].x, acc[a][b]);
          acc[a][b] = fmaf(v4[a].y, c4[b].y, acc[a][b]);
          acc[a][b] = fmaf(v4[a].z, c4[b].z, acc[a][b]);
          acc[a][b] = fmaf(v4[a].w, c4[b].w, acc[a][b]);
        }
    }
    float *dst = scr + (size_t)(g * T + mt) * 16;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) dst[a * 4 + b] = acc[a][b];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Mi * Nj; o += NT) {
    const int i = o % Mi, j = o / Mi;
    const int mt = (i >> 2) + (j >> 2) * ti, q = (i & 3) * 4 + (j & 3);
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += scr[(size_t)(g * T + mt) * 16 + q];
    W[i + (size_t)j * ldw] = (Cinit ? Cinit[i + (size_t)j * ldi] : 0.f) + s;
  }
  __syncthreads();
}

__device__ void gemm_nn_sub_f32(float *Cm, int ldc, const float *V, int ldv, const float *W, int ldw, int K, int Mi,
                                int Nj) {
  const int tk = K >> 2, tj = (Nj + 7) >> 3;
  for (int u = threadIdx.x; u < tk * tj; u += NT) {
    const int k0 = (u % tk) * 4, j0 = (u / tk) * 8, jn = min(8, Nj - j0);
    float4 acc[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[b] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < Mi; ++i) {
      const float4 v = *reinterpret_cast<const float4 *>(V + (size_t)i * ldv + k0);
      const float *w = W + i + (size_t)j0 * ldw;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float wb = b < jn ? w[(size_t)b * ldw] : 0.f;
        acc[b].x = fmaf(v.x, wb, acc[b].x);
        acc[b].y = fmaf(v.y, wb, acc[b].y);
        acc[b].z = fmaf(v.z, wb, acc[b].z);
        acc[b].w = fmaf(v.w, wb, acc[b].w);
      }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if (b < jn) {
        float4 *c = reinterpret_cast<float4 *>(Cm + (size_t)(j0 + b) * ldc + k0);
        float4 x = *c;
        x.x -= acc[b].x;
        x.y -= acc[b].y;
        x.z -= acc[b].z;
        x.w -= acc[b].w;
        *c = x;
      }
  }
  __syncthreads();
}

// W(i,j) = [Cinit(i,j)] + sum_{k<K} V(k,i) C(k,j), i < Mi, j < Nj.
// Short output sets split K among thread groups; partial sums are combined
// in a fixed order through `scr` (>= NT elements).
template <typename Real>
__device__ void gemm_tn(Real *W, int ldw, const Real *V, int ldv, const Real *Cm, int ldc, int K, int Mi,
                        int Nj, const Real *Cinit, int ldi, Real *scr) {
  const int O = Mi * Nj;
  if (O <= 0) return;
  if constexpr (sizeof(Real) == 4) {
    gemm_tn_f32(W, ldw, V, ldv, Cm, ldc, K, Mi, Nj, Cinit, ldi, scr);
    return;
  }
  const int tid = threadIdx.x;
  if (O >= NT / 2 || K < 64) {
    for (int o = tid; o < O; o += NT) {
      const int i = o % Mi, j = o / Mi;
      const Real *v = V + (size_t)i * ldv;
      const Real *c = Cm + (size_t)j * ldc;
      Real s0 = 0, s1 = 0;
      int k = 0;
      for (; k + 1 < K; k += 2) {
        s0 = fma(v[k], c[k], s0);
        s1 = fma(v[k + 1], c[k + 1], s1);
      }
      if (k < K) s0 = fma(v[k], c[k], s0);
      const Real base = Cinit ? Cinit[i + (size_t)j * ldi] : Real(0);
      W[i + (size_t)j * ldw] = base + (s0 + s1);
    }
    __syncthreads();
    return;
  }
  int G = NT / O;
  if (G > 16) G = 16;
  const int Kc = (K + G - 1) / G;
  const int o = tid % O, g = tid / O;
  if (g < G) {
    const int i = o % Mi, j = o / Mi;
    const Real *v = V + (size_t)i * ldv;
    const Real *c = Cm + (size_t)j * ldc;
    const int k0 = g * Kc, k1 = min(K, k0 + Kc);
    Real s = 0;
    for (int k = k0; k < k1; ++k) s = fma(v[k], c[k], s);
    scr[g * O + o] = s;
  }
  __syncthreads();
  if (tid < O) {
    const int i = tid % Mi, j = tid / Mi;
    Real s = 0;
    for (int q = 0; q < G; ++q) s += scr[q * O + tid];
    const Real base = Cinit ? Cinit[i + (size_t)j * ldi] : Real(0);
    W[i + (size_t)j * ldw] = base + s;
  }
  __syncthreads();
}

// C(k,j) -= sum_{i<Mi} V(k,i) W(i,j), k < K, j < Nj. Threads run along k.
// The FP64 version accumulates into C itself (C = fma(-V, W, C), terms in
// ascending i): a separate subtraction per output would cost the FP64 pipe
// as much as a DFMA, one extra operation per Mi (as few as 8) DFMAs.
template <typename Real>
__device__ void gemm_nn_sub(Real *Cm, int ldc, const Real *V, int ldv, const Real *W, int ldw, int K, int Mi,
                            int Nj) {
  if constexpr (sizeof(Real) == 4) {
    gemm_nn_sub_f32(Cm, ldc, V, ldv, W, ldw, K, Mi, Nj);
    return;
  }
  const int nchunk = (Nj + 7) / 8;
  const int total = K * nchunk;
  for (int it = threadIdx.x; it < total; it += NT) {
    const int k = it % K, jc = it / K;
    const int j0 = jc * 8, jn = min(8, Nj - j0);
    Real acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = q < jn ? Cm[k + (size_t)(j0 + q) * ldc] : Real(0);
    for (int i = 0; i < Mi; ++i) {
      const Real v = V[k + (size_t)i * ldv];
      const Real *w = W + i + (size_t)j0 * ldw;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < jn) acc[q] = fma(-v, w[(size_t)q * ldw], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < jn) Cm[k + (size_t)(j0 + q) * ldc] = acc[q];
  }
  __syncthreads();
}

// W <- T^T W (trans) or T W in place, T an ib x ib upper triangle (leading
// dimension ldq), ib even and <= 32. FP64: a group of ib / 2 lanes takes one
// column of W: lane h holds rows h and ib - 1 - h and forms both outputs from
// the group's values by shuffles, (h + 1) + (ib - h) = ib + 1 terms, one
// useful FMA per step (a lane per row would idle through half of its steps,
// and an idle FP64 step costs the FP64 pipe as much as a used one); terms of
// each output in ascending order.
template <typename Real>
__device__ void trmm_tw(Real *W, int ldw, const Real *Tq, int ldq, int ib, int Nj, int trans) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (sizeof(Real) == 4) {
    // FP32 (idle FMA steps are cheap there): one row per lane, lane i walking
    // the terms from its own offset so that a group's lanes read T from
    // different banks
    const int G = 32 / ib, grp = lane / ib, i = lane - grp * ib;
    for (int j0 = warp * G; j0 < Nj; j0 += NWARP * G) {
      const int j = j0 + grp;
      const bool on = grp < G && j < Nj;
      Real *w = W + (size_t)j * ldw;
      const Real wl = on ? w[i] : Real(0);
      Real s = 0;
      for (int u = 0; u < ib; ++u) {
        int l = i + u;
        if (l >= ib) l -= ib;
        const Real wv = __shfl_sync(0xffffffffu, wl, (grp * ib + l) & 31);
        if (on && (trans ? l <= i : l >= i)) s = fma(trans ? Tq[l + (size_t)i * ldq] : Tq[i + (size_t)l * ldq], wv, s);
      }
      __syncwarp();
      if (on) w[i] = s;
    }
    __syncthreads();
    return;
  }
  const int hb = ib / 2, G = 32 / hb, grp = lane / hb, h = lane - grp * hb;
  const int ra = h, rb = ib - 1 - h;
  for (int j0 = warp * G; j0 < Nj; j0 += NWARP * G) {
    const int j = j0 + grp;
    const bool on = grp < G && j < Nj;
    Real *w = W + (size_t)j * ldw;
    const Real wa = on ? w[ra] : Real(0), wb = on ? w[rb] : Real(0);
    Real sa = 0, sb = 0;
    for (int u = 0; u <= ib; ++u) {
      // output row r of this step and its source row l (trans: l <= r; else l >= r)
      const bool first = trans ? u <= h : u < ib - h;
      const int l = trans ? (first ? u : u - h - 1) : (first ? h + u : u - 1);
      const int r = first ? ra : rb;
      const int src = grp * hb + (l < hb ? l : ib - 1 - l);
      const Real xa = __shfl_sync(0xffffffffu, wa, src & 31);
      const Real xb = __shfl_sync(0xffffffffu, wb, src & 31);
      const Real c = trans ? Tq[l + (size_t)r * ldq] : Tq[r + (size_t)l * ldq];
      Real acc = first ? sa : sb;
      acc = fma(c, l < hb ? xa : xb, acc);
      if (first)
        sa = acc;
      else
        sb = acc;
    }
    __syncwarp();
    if (on) {
      w[ra] = sa;
      w[rb] = sb;
    }
  }
  __syncthreads();
}

// Ct(i,j) -= W(i,j): the identity top block of TS/TT reflectors.
template <typename Real>
__device__ void sub_top(Real *Ct, int ldt, const Real *W, int ldw, int Mi, int Nj) {
  for (int o = threadIdx.x; o < Mi * Nj; o += NT) {
    const int i = o % Mi, j = o / Mi;
    Ct[i + (size_t)j * ldt] -= W[i + (size_t)j * ldw];
  }
  __syncthreads();
}

enum { PANEL_GE = 0, PANEL_TS = 1, PANEL_TT = 2 };

// Householder factorization of one block of ib columns held in shared memory.
//  GE: P is L x ib, column jj has alpha = P(jj,jj) and x2 = P(jj+1:L, jj).
//  TS: alpha = Rt(jj,jj), x2 = P(0:L, jj) (the killed square tile).
//  TT: alpha = Rt(jj,jj), x2 = P(0:q0+jj+1, jj) (upper-triangular tile).
// On return P holds the reflectors' lower parts (GE: R above) and sh.tau the
// scalars; Rt's upper triangle holds the updated R rows of the block.
template <typename Real>
__device__ void factor_block(int mode, Real *P, int ld, int L, int ib, Real *Rt, int ldt, int q0,
                             Shared<Real> &sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int jj = 0; jj < ib; ++jj) {
    const int r0 = (mode == PANEL_GE) ? jj + 1 : 0;
    const int r1 = (mode == PANEL_TT) ? min(L, q0 + jj + 1) : L;
    Real *col = P + (size_t)jj * ld;
    const int nact = min(NT, r1 - r0);  // threads holding rows of the column
    Real ss = 0;
    for (int k = r0 + tid; k < r1; k += NT) ss = fma(col[k], col[k], ss);
    ss = block_sum(ss, sh, nact);
    Real snorm;
    const bool plain = ss > RealTraits<Real>::tiny && ss < RealTraits<Real>::huge;
    if constexpr (sizeof(Real) == 8) {
      // FP64: the norm only matters to thread 0 below, which forms ||(alpha, x)|| from ss itself
      // (a warp-wide square root on every warp would occupy the FP64 pipe for nothing)
      snorm = plain ? ss : Real(0);
    }
    if (plain) {
      if constexpr (sizeof(Real) == 4) snorm = sqrt(ss);
    } else {
      Real am = 0;
      for (int k = r0 + tid; k < r1; k += NT) am = fmax(am, fabs(col[k]));
      am = block_max(am, sh, nact);
      if (am == Real(0)) {
        snorm = 0;
      } else {
        const Real inv = Real(1) / am;
        Real s2 = 0;
        for (int k = r0 + tid; k < r1; k += NT) {
          const Real x = col[k] * inv;
          s2 = fma(x, x, s2);
        }
        s2 = block_sum(s2, sh, nact);
        snorm = am * sqrt(s2);
      }
    }
    Real *diag = (mode == PANEL_GE) ? &col[jj] : &Rt[jj + (size_t)jj * ldt];
    if (tid == 0) {
      const Real alpha = *diag;
      Real beta = alpha, t = 0, scale = 0;
      if (snorm != Real(0)) {
        Real h;
        if constexpr (sizeof(Real) == 8)  // unscaled: snorm holds ss; sqrt(alpha^2 + ss) cannot overflow
          h = plain ? (fabs(alpha) < 1e150 ? sqrt(fma(alpha, alpha, ss)) : hypot(alpha, sqrt(ss)))
                    : hypot(alpha, snorm);
        else
          h = hypot(alpha, snorm);
        beta = (alpha >= Real(0)) ? -h : h;
        t = (beta - alpha) / beta;
        scale = Real(1) / (alpha - beta);
      }
      *diag = beta;
      sh.tau[jj] = t;
      sh.bc[0] = t;
      sh.bc[1] = scale;
    }
    __syncthreads();
    const Real t = sh.bc[0], scale = sh.bc[1];
    for (int k = r0 + tid; k < r1; k += NT) col[k] *= scale;
    __syncthreads();
    if (t == Real(0)) continue;  // identity reflector: nothing to apply
    // w_c = top(jj,c) + v^T P(:,c) for the block's later columns; short columns share a warp
    // (LPC lanes per column, 32 / LPC columns per warp), which saves shuffle-add levels
    const int nr = r1 - r0, ncl = ib - jj - 1;
    const int LPC = nr > 64 ? 32 : (nr > 32 ? 16 : 8), CPW = 32 / LPC;
    const int sub = lane / LPC, sl = lane - sub * LPC;
    for (int cw0 = jj + 1 + warp * CPW; cw0 < ib; cw0 += NWARP * CPW) {
      const int c = cw0 + sub;
      const bool on = c < ib;
      const Real *pc = P + (size_t)(on ? c : jj) * ld;
      Real s = 0;
      if (on)
        for (int k = r0 + sl; k < r1; k += LPC) s = fma(col[k], pc[k], s);
      for (int o = LPC >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (on && sl == 0) {
        const Real top = (mode == PANEL_GE) ? pc[jj] : Rt[jj + (size_t)c * ldt];
        sh.wv[c] = t * (top + s);
      }
    }
    __syncthreads();
    for (int e = tid; e < nr * ncl; e += NT) {
      const int c = jj + 1 + e / nr, k = r0 + e % nr;
      Real *pc = P + (size_t)c * ld;
      pc[k] = fma(-col[k], sh.wv[c], pc[k]);
    }
    if (tid > jj && tid < ib) {
      if (mode == PANEL_GE)
        P[jj + (size_t)tid * ld] -= sh.wv[tid];
      else
        Rt[jj + (size_t)tid * ldt] -= sh.wv[tid];
    }
    __syncthreads();
  }
}

// T of a block from the Gram matrix G = V^T V (only G(l, j), l < j, used).
template <typename Real>
__device__ void build_t(Real *Tq, int ldq, const Real *G, int ib, const Shared<Real> &sh) {
  for (int e = threadIdx.x; e < ib * ldq; e += NT) Tq[e] = 0;
  __syncthreads();
  for (int jj = 0; jj < ib; ++jj) {
    const int tid = threadIdx.x;
    if (tid < jj) {
      Real y = 0;
      for (int l = tid; l < jj; ++l) y = fma(Tq[tid + (size_t)l * ldq], G[l + (size_t)jj * ib], y);
      Tq[tid + (size_t)jj * ldq] = -sh.tau[jj] * y;
    } else if (tid == jj) {
      Tq[jj + (size_t)jj * ldq] = sh.tau[jj];
    }
    __syncthreads();
  }
}

// Set the structural zeros (and unit diagonal) of a staged V chunk.
//  GE: unit lower; chunk column cc is global block column coff + cc, local
//      row kl is block row kl: zero above, one on the diagonal.
//  TT: upper triangular: zero below row roff + coff + cc.
template <typename Real>
__device__ void shape_v(Real *V, int ld, int L, int ncols, int mode, int coff, int roff) {
  for (int e = threadIdx.x; e < L * ncols; e += NT) {
    const int c = e / L, k = e - c * L;
    Real *x = V + (size_t)c * ld + k;
    if (mode == PANEL_GE) {
      if (k < coff + c)
        *x = 0;
      else if (k == coff + c)
        *x = 1;
    } else if (mode == PANEL_TT) {
      if (k > roff + coff + c) *x = 0;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------- task bodies --

template <typename Real>
__host__ __device__ inline size_t engine_smem_bytes(int nb, int ib, int w, int wt, int vc);

// Updates UNMQR / TSMQR / TTMQR of one column slab (also used for Q and Q^T
// applied to right-hand-side blocks). V is staged in chunks of columns; the
// chunk buffer comes last in shared memory and may use what the panel tasks
// need beyond the updates: in FP64, a block of L reflector rows (GE and TT
// blocks get shorter towards one end of the tile) takes chunks as wide as
// fit (8, 16 or 32 columns, column stride L + pad), so a short block needs
// fewer staging rounds, and none for its second product when one chunk
// holds all of it.
template <typename Real>
__device__ void task_update(const EngineParams &p, const Geo<Real> &g, const Task &t, Shared<Real> &sh,
                            Real *dyn, uint32_t &phase) {
  const int nb = g.nb, ib = g.ib, lds = g.lds, cw = t.cw;
  const int wmax = t.tgt == 0 ? g.w : g.wb;
  const int VC = g.vc;
  Real *C1 = dyn;
  Real *C2 = C1 + (size_t)lds * wmax;
  const int ldq = sizeof(Real) == 8 ? g.ldt : ib;  // T of the block (FP64: padded for the paired trmm)
  Real *Tq = C2 + (size_t)lds * wmax;
  Real *W = Tq + (size_t)ib * ldq;
  Real *scr = W + (size_t)ib * wmax;
  const size_t su = (sizeof(Real) == 4 ? 4 : 1) * (size_t)(((VC + 3) / 4) * ((wmax + 3) / 4) * 16);
  Real *Vc = scr + (su > (size_t)NT ? su : (size_t)NT);
  const size_t vcap = engine_smem_bytes<Real>(nb, ib, g.w > g.wb ? g.w : g.wb, g.wt, VC) / sizeof(Real) -
                      (size_t)(Vc - dyn);
  const int op = t.op;
  const bool pair = op != OP_UNMQR;
  const int mode = op == OP_UNMQR ? PANEL_GE : (op == OP_TSMQR ? PANEL_TS : PANEL_TT);
  Real *g1 = g.target(t, pair ? t.r : t.i);
  Real *g2 = pair ? g.target(t, t.i) : nullptr;
  const Real *Vt = g.tile(t.i, t.k);
  const Real *Tt = g.tfac(pair ? 1 : 0, t.i, t.k);
  {
    Copy<Real> cp[2] = {{C1, lds, g1, nb, nb, cw}, {C2, lds, g2, nb, pair ? nb : 0, cw}};
    stage(p, sh, cp, 2, phase);
  }
  const int nq = nb / ib;
  for (int qq = 0; qq < nq; ++qq) {
    const int q = t.trans ? qq : nq - 1 - qq;
    if (t.blk > 0 && q != t.blk - 1) continue;  // one block of a split panel, on the panel's own tiles
    const int q0 = q * ib;
    const int vr0 = (mode == PANEL_GE) ? q0 : 0;
    const int L = (mode == PANEL_GE) ? nb - q0 : (mode == PANEL_TS ? nb : q0 + ib);
    Real *Cb = (mode == PANEL_GE) ? C1 + q0 : C2;
    Real *Ct = C1 + q0;
    int vq = VC, ldv = lds;
    if constexpr (sizeof(Real) == 8) {
      ldv = L + smem_pad<Real>();
      while (2 * vq <= ib && ib % (2 * vq) == 0 && (size_t)ldv * 2 * vq <= vcap) vq *= 2;
    }
    const int nchunk = ib / vq;
    for (int c = 0; c < nchunk; ++c) {
      __syncthreads();
      Copy<Real> cp[2] = {{Vc, ldv, Vt + (size_t)(q0 + c * vq) * nb + vr0, nb, L, vq},
                          {Tq, ldq, Tt + (size_t)q * ib * ib, ib, c == 0 ? ib : 0, ib}};
      stage(p, sh, cp, 2, phase);
      shape_v(Vc, ldv, L, vq, mode, c * vq, q0);
      gemm_tn(W + c * vq, ib, Vc, ldv, Cb, lds, L, vq, cw, pair ? Ct + c * vq : nullptr, lds, scr);
    }
    trmm_tw(W, ib, Tq, ldq, ib, cw, t.trans);
    if (pair) sub_top(Ct, lds, W, ib, ib, cw);
    for (int c = 0; c < nchunk; ++c) {
      if (nchunk > 1) {
        __syncthreads();
        Copy<Real> cp[1] = {{Vc, ldv, Vt + (size_t)(q0 + c * vq) * nb + vr0, nb, L, vq}};
        stage(p, sh, cp, 1, phase);
        shape_v(Vc, ldv, L, vq, mode, c * vq, q0);
      }
      gemm_nn_sub(Cb, lds, Vc, ldv, W + c * vq, ib, L, vq, cw);
    }
  }
  store_cols(g1, nb, C1, lds, nb, cw, 0, 0);
  if (pair) store_cols(g2, nb, C2, lds, nb, cw, 0, 0);
}

// GEQRT (mode GE), TSQRT (TS) and TTQRT (TT) of one tile (pair).
template <typename Real>
__device__ void task_panel(const EngineParams &p, const Geo<Real> &g, const Task &t, Shared<Real> &sh,
                           Real *dyn, uint32_t &phase) {
  const int nb = g.nb, ib = g.ib, lds = g.lds, wt = g.wt, ldt = g.ldt;
  const int mode = t.op == OP_GEQRT ? PANEL_GE : (t.op == OP_TSQRT ? PANEL_TS : PANEL_TT);
  Real *P = dyn;
  Real *Rt = P + (size_t)lds * ib;
  const int ldq = sizeof(Real) == 8 ? ldt : ib;  // T of the block (FP64: padded for the paired trmm)
  Real *Tq = Rt + (size_t)ldt * ib;
  Real *Ct = Tq + (size_t)ib * ldq;
  Real *Cb = Ct + (size_t)ldt * wt;
  Real *G = Cb;  // the Gram matrix is dead before the trailing slabs use Cb
  Real *W = Cb + (size_t)(lds * wt > ib * ib ? lds * wt : ib * ib);
  Real *scr = W + (size_t)ib * wt;
  Real *XR = g.tile(t.r, t.k);  // GE: the tile itself (r == i)
  Real *XB = g.tile(t.i, t.k);
  Real *Tg = g.tfac(mode == PANEL_GE ? 0 : 1, t.i, t.k);
  const int nq = nb / ib;
  // a block task of a split panel factors its block only; separate update tasks apply it to the
  // trailing slabs
  const int qa = t.blk > 0 ? t.blk - 1 : 0, qb = t.blk > 0 ? t.blk : nq;
  for (int q = qa; q < qb; ++q) {
    const int q0 = q * ib;
    const int L = (mode == PANEL_GE) ? nb - q0 : (mode == PANEL_TS ? nb : q0 + ib);
    const int br0 = (mode == PANEL_GE) ? q0 : 0;  // first tile row held in P
    __syncthreads();
    {
      Copy<Real> cp[2] = {{P, lds, XB + (size_t)q0 * nb + br0, nb, L, ib},
                          {Rt, ldt, XR + (size_t)q0 * nb + q0, nb, mode == PANEL_GE ? 0 : ib, ib}};
      stage(p, sh, cp, 2, phase);
    }
    if (mode == PANEL_TT) {  // the strict lower part of R2's tile is GEQRT's V, not data
      for (int e = threadIdx.x; e < L * ib; e += NT) {
        const int c = e / L, k = e - c * L;
        if (k > q0 + c) P[(size_t)c * lds + k] = 0;
      }
      __syncthreads();
    }
    factor_block(mode, P, lds, L, ib, Rt, ldt, q0, sh);
    // write back the factored block
    if (mode == PANEL_GE) {
      store_cols(XB + (size_t)q0 * nb + q0, nb, P, lds, L, ib, 0, 0);
    } else {
      store_cols(XR + (size_t)q0 * nb + q0, nb, Rt, ldt, ib, ib, 1, 0);
      store_cols(XB + (size_t)q0 * nb, nb, P, lds, L, ib, mode == PANEL_TT ? 1 : 0, q0);
    }
    __syncthreads();
    if (mode == PANEL_GE) shape_v(P, lds, L, ib, PANEL_GE, 0, 0);
    gemm_tn(G, ib, P, lds, P, lds, L, ib, ib, (const Real *)nullptr, 0, scr);
    build_t(Tq, ldq, G, ib, sh);
    store_cols(Tg + (size_t)q * ib * ib, ib, Tq, ldq, ib, ib, 0, 0);
    if (t.blk > 0) break;
    // trailing columns of the tile(s): block reflector applied with Q^T
    for (int c0 = q0 + ib; c0 < nb; c0 += wt) {
      const int wc = min(wt, nb - c0);
      __syncthreads();
      if (mode == PANEL_GE) {
        Copy<Real> cp[1] = {{Cb, lds, XB + (size_t)c0 * nb + q0, nb, L, wc}};
        stage(p, sh, cp, 1, phase);
        gemm_tn(W, ib, P, lds, Cb, lds, L, ib, wc, (const Real *)nullptr, 0, scr);
        trmm_tw(W, ib, Tq, ldq, ib, wc, 1);
        gemm_nn_sub(Cb, lds, P, lds, W, ib, L, ib, wc);
        store_cols(XB + (size_t)c0 * nb + q0, nb, Cb, lds, L, wc, 0, 0);
      } else {
        Copy<Real> cp[2] = {{Ct, ldt, XR + (size_t)c0 * nb + q0, nb, ib, wc},
                            {Cb, lds, XB + (size_t)c0 * nb, nb, L, wc}};
        stage(p, sh, cp, 2, phase);
        gemm_tn(W, ib, P, lds, Cb, lds, L, ib, wc, (const Real *)Ct, ldt, scr);
        trmm_tw(W, ib, Tq, ldq, ib, wc, 1);
        sub_top(Ct, ldt, W, ib, ib, wc);
        gemm_nn_sub(Cb, lds, P, lds, W, ib, L, ib, wc);
        store_cols(XR + (size_t)c0 * nb + q0, nb, Ct, ldt, ib, wc, 0, 0);
        store_cols(XB + (size_t)c0 * nb, nb, Cb, lds, L, wc, 0, 0);
      }
    }
  }
}

// ------------------------------------------------------ FP64 vector tasks --
// Compensated products and sums (TwoProduct with FMA, TwoSum of Knuth): the
// residual and A^T r of the refinement are accumulated as in twice the
// working precision (Ogita, Rump, Oishi 2005, "Dot2").

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
  s = a + b;
  const double z = s - a;
  e = (a - (s - z)) + (b - z);
}

// (s, c) += a * x
__device__ __forceinline__ void dot2_step(double a, double x, double &s, double &c) {
  const double p = a * x;
  const double ep = fma(a, x, -p);
  double t, es;
  two_sum(s, p, t, es);
  s = t;
  c += ep + es;
}

// (s1, c1) += (s2, c2)
__device__ __forceinline__ void dot2_merge(double &s1, double &c1, double s2, double c2) {
  double t, e;
  two_sum(s1, s2, t, e);
  s1 = t;
  c1 += c2 + e;
}

// sum over q = q0, q0 + step, ... < q1 of M(q, o) g_q (transposed) or M(o, q) g_q, M column-major
// with leading dimension ld (in shared memory when staged, else global: M is final for the whole
// launch, R tiles after their factorization, the inverses after their TRINV task), in FP64 with
// four chains. In the transposed walk every thread reads its own column, so each starts at its
// own offset (the lane index, cyclically): the lanes of a warp then read different rows and
// shared-memory banks. The order of the terms depends only on (o, q0, q1, step), never on where
// M is, so staged and unstaged runs give the same bits.
template <typename M>
__device__ __forceinline__ double tile_dot(const M *m, int ld, bool transposed, int o, int q0, int q1, int step,
                                           const double *g) {
  const int K = q1 > q0 ? (q1 - q0 + step - 1) / step : 0;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (transposed) {
    const M *col = m + (size_t)o * ld;
    int k = K > 0 ? (o & 31) % K : 0;
    auto term = [&](double acc) {
      const int q = q0 + k * step;
      acc = fma(ptx::to_f64(col[q]), g[q], acc);
      if (++k == K) k = 0;
      return acc;
    };
    int c = 0;
    for (; c + 3 < K; c += 4) {
      a0 = term(a0);
      a1 = term(a1);
      a2 = term(a2);
      a3 = term(a3);
    }
    for (; c < K; ++c) a0 = term(a0);
  } else {
    const M *row = m + o;
    const size_t qs = (size_t)step * ld;
    const M *p = row + (size_t)q0 * ld;
    const double *gq = g + q0;
    int c = 0;
    for (; c + 3 < K; c += 4, p += 4 * qs, gq += 4 * step) {
      a0 = fma(ptx::to_f64(p[0]), gq[0], a0);
      a1 = fma(ptx::to_f64(p[qs]), gq[step], a1);
      a2 = fma(ptx::to_f64(p[2 * qs]), gq[2 * step], a2);
      a3 = fma(ptx::to_f64(p[3 * qs]), gq[3 * step], a3);
    }
    for (; c < K; ++c, p += qs, gq += step) a0 = fma(ptx::to_f64(p[0]), gq[0], a0);
  }
  return (a0 + a1) + (a2 + a3);
}

__device__ __forceinline__ bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// Byte offset of the tiles a triangular-solve step stages in shared memory
// (after g_i and the partial sums: nb + NT doubles at most).
constexpr uint32_t kVecStageOff = 4096;
static_assert((128 + NT) * 8 <= kVecStageOff, "vector scratch overlaps the staged tiles");

// KU: elements of A each thread keeps in flight in the residual and A^T r
// loops (16 in the one-CTA-per-SM tensor-core kernel, 8 where two CTAs share
// an SM's registers).
template <typename Real, int KU>
__device__ void task_vector(const EngineParams &p, const Problem &P, const Geo<Real> &g, const Task &t,
                            double *sm, Shared<Real> &sh, uint32_t &phase) {
  const int nb = g.nb, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Real *A0 = (const Real *)P.A0;
  // a round of a tolerance-stopped refinement: nothing to do once an earlier round met the
  // tolerance (the x updates and checks are ordered after the check that decided it; the
  // other tasks of the round right after it may read the flag early or late, and only
  // write scratch vectors that no later task reads)
  const bool tolm = t.trans == 2;
  bool comp = t.tgt != 0;  // residual and A^T r: compensated (Dot2) or plain FP64 sums
  if (t.op == OP_RGATE) {
    // gate of round k: if the refinement stopped at round k - 2 or earlier, no task of rounds >= k
    // may run; they all follow this gate, so it releases none of its successors and counts them
    // (t.j tasks) as done
    if (tid == 0) {
      const int conv = __ldcg(&P.rs->conv);
      if (conv != 0 && t.k >= conv + 1) {
        sh.norelease = 1;
        atomicAdd(&p.ctl->done.v, (unsigned)t.j);
      }
    }
    __syncthreads();
    return;
  }
  if (tolm) {  // one thread reads the state, so that the whole CTA takes the same branch
    if (tid == 0) {
      const int conv = __ldcg(&P.rs->conv);
      sh.vskip = conv != 0 && t.k >= conv;
      sh.vcomp = __ldcg(&P.rs->mode[t.k]) != 0;
    }
    __syncthreads();
    if (sh.vskip) return;
    comp = sh.vcomp != 0;
  }
  switch (t.op) {
    case OP_RESID: {  // partial sums of A(rows of tile i, columns of chunk t.j) x
      const int r0 = t.i * nb, nr = min(nb, P.M - r0);
      const int clo = t.j * kResChunk * nb, chi = min(P.N, clo + kResChunk * nb);
      const int G = NT / nb;  // column groups
      const int rr = tid % nb, gi = tid / nb;
      double s = 0.0, c = 0.0;
      if (rr < nr && gi < G && !comp) {  // plain FP64 round: four independent FMA chains
        const Real *arow = A0 + r0 + rr;
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = clo + gi;
        // KU columns in flight per thread (the loads of A are the latency to hide); each chain
        // takes its terms in the same order as one step at a time
        for (; j + (KU - 1) * G < chi; j += KU * G) {
          Real a[KU];
          double xv[KU];
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            a[u] = __ldcg(arow + (long long)(j + u * G) * P.lda0);
            xv[u] = __ldcg(P.x + j + u * G);
          }
#pragma unroll
          for (int u = 0; u < KU; u += 4) {
            s = fma(ptx::to_f64(a[u]), xv[u], s);
            s1 = fma(ptx::to_f64(a[u + 1]), xv[u + 1], s1);
            s2 = fma(ptx::to_f64(a[u + 2]), xv[u + 2], s2);
            s3 = fma(ptx::to_f64(a[u + 3]), xv[u + 3], s3);
          }
        }
        for (; j + 3 * G < chi; j += 4 * G) {
          s = fma(ptx::to_f64(__ldcg(arow + (long long)j * P.lda0)), __ldcg(P.x + j), s);
          s1 = fma(ptx::to_f64(__ldcg(arow + (long long)(j + G) * P.lda0)), __ldcg(P.x + j + G), s1);
          s2 = fma(ptx::to_f64(__ldcg(arow + (long long)(j + 2 * G) * P.lda0)), __ldcg(P.x + j + 2 * G), s2);
          s3 = fma(ptx::to_f64(__ldcg(arow + (long long)(j + 3 * G) * P.lda0)), __ldcg(P.x + j + 3 * G), s3);
        }
        for (; j < chi; j += G) s = fma(ptx::to_f64(__ldcg(arow + (long long)j * P.lda0)), __ldcg(P.x + j), s);
        s = (s + s1) + (s2 + s3);
      } else if (rr < nr && gi < G) {
        // four independent compensated sums (more FP64 work in flight), merged in a fixed order
        const Real *arow = A0 + r0 + rr;
        double s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0, s3 = 0.0, c3 = 0.0;
        int j = clo + gi;
        for (; j + (KU - 1) * G < chi; j += KU * G) {  // KU columns in flight, the same order per sum
          Real a[KU];
          double xv[KU];
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            a[u] = __ldcg(arow + (long long)(j + u * G) * P.lda0);
            xv[u] = __ldcg(P.x + j + u * G);
          }
#pragma unroll
          for (int u = 0; u < KU; u += 4) {
            dot2_step(ptx::to_f64(a[u]), xv[u], s, c);
            dot2_step(ptx::to_f64(a[u + 1]), xv[u + 1], s1, c1);
            dot2_step(ptx::to_f64(a[u + 2]), xv[u + 2], s2, c2);
            dot2_step(ptx::to_f64(a[u + 3]), xv[u + 3], s3, c3);
          }
        }
        for (; j + 3 * G < chi; j += 4 * G) {
          const double a0 = ptx::to_f64(__ldcg(arow + (long long)j * P.lda0));
          const double a1 = ptx::to_f64(__ldcg(arow + (long long)(j + G) * P.lda0));
          const double a2 = ptx::to_f64(__ldcg(arow + (long long)(j + 2 * G) * P.lda0));
          const double a3 = ptx::to_f64(__ldcg(arow + (long long)(j + 3 * G) * P.lda0));
          dot2_step(a0, __ldcg(P.x + j), s, c);
          dot2_step(a1, __ldcg(P.x + j + G), s1, c1);
          dot2_step(a2, __ldcg(P.x + j + 2 * G), s2, c2);
          dot2_step(a3, __ldcg(P.x + j + 3 * G), s3, c3);
        }
        for (; j < chi; j += G) dot2_step(ptx::to_f64(__ldcg(arow + (long long)j * P.lda0)), __ldcg(P.x + j), s, c);
        dot2_merge(s, c, s1, c1);
        dot2_merge(s2, c2, s3, c3);
        dot2_merge(s, c, s2, c2);
      }
      sm[tid] = s;
      sm[NT + tid] = c;
      __syncthreads();
      if (tid < nr) {
        double S = sm[tid], C = sm[NT + tid];
        for (int q = 1; q < G; ++q) dot2_merge(S, C, sm[q * nb + tid], sm[NT + q * nb + tid]);
        const size_t mp = (size_t)g.m * nb;
        P.rp[2 * ((size_t)t.j * mp + r0 + tid)] = S;
        P.rp[2 * ((size_t)t.j * mp + r0 + tid) + 1] = C;
      }
      __syncthreads();
      break;
    }
    case OP_RESR: {  // r_i = b_i - sum of the column-chunk partials, in chunk order
      const int r0 = t.i * nb, nr = min(nb, P.M - r0);
      const int nrc = (g.n + kResChunk - 1) / kResChunk;
      const size_t mp = (size_t)g.m * nb;
      for (int rr = tid; rr < nr; rr += NT) {
        double S = __ldcg(P.rp + 2 * (size_t)(r0 + rr)), C = __ldcg(P.rp + 2 * (size_t)(r0 + rr) + 1);
        for (int q = 1; q < nrc; ++q)
          dot2_merge(S, C, __ldcg(P.rp + 2 * ((size_t)q * mp + r0 + rr)), __ldcg(P.rp + 2 * ((size_t)q * mp + r0 + rr) + 1));
        double u, e2;
        two_sum(__ldcg(P.b + r0 + rr), -S, u, e2);
        P.r[r0 + rr] = u + (e2 - C);
      }
      break;
    }
    case OP_TRINV: {  // inverse of the upper-triangular leading n_i x n_i part of R_ii (thread per column)
      const int i = t.i, n_i = min(nb, P.N - i * nb);
      const Real *R = g.tile(i, i);
      double *X = P.rinv + (size_t)i * nb * nb;
      for (int e = tid; e < nb * nb; e += NT) X[e] = 0.0;
      __syncthreads();
      for (int j = tid; j < n_i; j += NT) {
        double *xj = X + (size_t)j * nb;
        const double djj = (double)__ldcg(R + (size_t)j * nb + j);
        if (djj == 0.0) {
          atomicExch(P.status, HQR_ERR_SINGULAR);
          if (P.rs) atomicMax(&P.rs->sing, ~(unsigned)(i * nb + j));
          continue;
        }
        xj[j] = 1.0 / djj;
        for (int k = j - 1; k >= 0; --k) {
          double s = 0.0;
          for (int l = k + 1; l <= j; ++l) s = fma((double)__ldcg(R + (size_t)l * nb + k), xj[l], s);
          const double dkk = (double)__ldcg(R + (size_t)k * nb + k);
          if (dkk == 0.0) {
            atomicExch(P.status, HQR_ERR_SINGULAR);
            if (P.rs) atomicMax(&P.rs->sing, ~(unsigned)(i * nb + k));
            break;
          }
          xj[k] = -s / dkk;
        }
      }
      break;
    }
    case OP_ATR: {  // partial sums of A(rows of chunk t.i, tile j)^T r
      const int c0 = t.j * nb, nc = min(nb, P.N - c0);
      const int rlo = t.i * kAtrChunk * nb, rhi = min(P.M, rlo + kAtrChunk * nb);
      const size_t np = (size_t)g.n * nb;
      for (int cc = warp; cc < nc; cc += NWARP) {
        const Real *acol = A0 + (long long)(c0 + cc) * P.lda0;
        double s = 0.0, c = 0.0, s1 = 0.0, c1 = 0.0, s2 = 0.0, c2 = 0.0, s3 = 0.0, c3 = 0.0;
        int i = rlo + lane;
        if (!comp) {  // plain FP64 round: FMA chains, then a plain warp sum
          for (; i + 32 * (KU - 1) < rhi; i += 32 * KU) {  // KU rows in flight, the same order per chain
            Real a[KU];
            double rv[KU];
#pragma unroll
            for (int u = 0; u < KU; ++u) {
              a[u] = __ldcg(acol + i + 32 * u);
              rv[u] = __ldcg(P.r + i + 32 * u);
            }
#pragma unroll
            for (int u = 0; u < KU; u += 4) {
              s = fma(ptx::to_f64(a[u]), rv[u], s);
              s1 = fma(ptx::to_f64(a[u + 1]), rv[u + 1], s1);
              s2 = fma(ptx::to_f64(a[u + 2]), rv[u + 2], s2);
              s3 = fma(ptx::to_f64(a[u + 3]), rv[u + 3], s3);
            }
          }
          for (; i + 96 < rhi; i += 128) {
            s = fma(ptx::to_f64(__ldcg(acol + i)), __ldcg(P.r + i), s);
            s1 = fma(ptx::to_f64(__ldcg(acol + i + 32)), __ldcg(P.r + i + 32), s1);
            s2 = fma(ptx::to_f64(__ldcg(acol + i + 64)), __ldcg(P.r + i + 64), s2);
            s3 = fma(ptx::to_f64(__ldcg(acol + i + 96)), __ldcg(P.r + i + 96), s3);
          }
          for (; i < rhi; i += 32) s = fma(ptx::to_f64(__ldcg(acol + i)), __ldcg(P.r + i), s);
          s = warp_sum((s + s1) + (s2 + s3));
          if (lane == 0) {
            P.gp[2 * ((size_t)t.i * np + c0 + cc)] = s;
            P.gp[2 * ((size_t)t.i * np + c0 + cc) + 1] = 0.0;
          }
          continue;
        }
        for (; i + 32 * (KU - 1) < rhi; i += 32 * KU) {  // KU rows in flight, the same order per sum
          Real a[KU];
          double rv[KU];
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            a[u] = __ldcg(acol + i + 32 * u);
            rv[u] = __ldcg(P.r + i + 32 * u);
          }
#pragma unroll
          for (int u = 0; u < KU; u += 4) {
            dot2_step(ptx::to_f64(a[u]), rv[u], s, c);
            dot2_step(ptx::to_f64(a[u + 1]), rv[u + 1], s1, c1);
            dot2_step(ptx::to_f64(a[u + 2]), rv[u + 2], s2, c2);
            dot2_step(ptx::to_f64(a[u + 3]), rv[u + 3], s3, c3);
          }
        }
        for (; i + 96 < rhi; i += 128) {  // four independent compensated sums, merged in a fixed order
          const double a0 = ptx::to_f64(__ldcg(acol + i)), a1 = ptx::to_f64(__ldcg(acol + i + 32));
          const double a2 = ptx::to_f64(__ldcg(acol + i + 64)), a3 = ptx::to_f64(__ldcg(acol + i + 96));
          dot2_step(a0, __ldcg(P.r + i), s, c);
          dot2_step(a1, __ldcg(P.r + i + 32), s1, c1);
          dot2_step(a2, __ldcg(P.r + i + 64), s2, c2);
          dot2_step(a3, __ldcg(P.r + i + 96), s3, c3);
        }
        for (; i < rhi; i += 32) dot2_step(ptx::to_f64(__ldcg(acol + i)), __ldcg(P.r + i), s, c);
        dot2_merge(s, c, s1, c1);
        dot2_merge(s2, c2, s3, c3);
        dot2_merge(s, c, s2, c2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
          dot2_merge(s, c, s2, c2);
        }
        if (lane == 0) {
          P.gp[2 * ((size_t)t.i * np + c0 + cc)] = s;
          P.gp[2 * ((size_t)t.i * np + c0 + cc) + 1] = c;
        }
      }
      break;
    }
    case OP_ATRR: {  // g_j = sum of the chunk partials, in chunk order
      const int c0 = t.j * nb, nc = min(nb, P.N - c0);
      const int nch = (g.m + kAtrChunk - 1) / kAtrChunk;
      const size_t np = (size_t)g.n * nb;
      for (int cc = tid; cc < nc; cc += NT) {
        double s = __ldcg(P.gp + 2 * (size_t)(c0 + cc)), c = __ldcg(P.gp + 2 * (size_t)(c0 + cc) + 1);
        for (int q = 1; q < nch; ++q)
          dot2_merge(s, c, __ldcg(P.gp + 2 * ((size_t)q * np + c0 + cc)), __ldcg(P.gp + 2 * ((size_t)q * np + c0 + cc) + 1));
        P.g[c0 + cc] = s + c;
      }
      break;
    }
    case OP_TRSV_TD:
    case OP_TRSV_D:
    case OP_TRSV_TU:
    case OP_TRSV_U: {
      // Triangular-solve steps with one tile: TD g_i <- X^T g_i, D g_i <- X g_i (X = R_ii^{-1}, FP64),
      // TU g_j -= R(i,j)^T g_i (j > i), U g_j -= R(j,i) g_i (j < i). g_i is staged once; every thread
      // owns one output (and half of its sum) and keeps four independent FP64 chains, with no FP64
      // cross-lane reductions (a warp-wide FP64 operation takes 16 cycles of the FP64 pipe).
      const int i = t.i, n_i = min(nb, P.N - i * nb);
      const bool diag = t.op == OP_TRSV_TD || t.op == OP_TRSV_D;
      const bool transposed = t.op == OP_TRSV_TD || t.op == OP_TRSV_TU;
      const int j = diag ? i : t.j;
      const int n_out = min(nb, P.N - j * nb);
      double *gi = P.g + (size_t)i * nb;
      double *go = P.g + (size_t)j * nb;
      double *gs = sm;         // g_i
      double *part = sm + nb;  // partial sums, (NT / nb) x nb
      // the step's tiles (R(i, j) or R(j, i); the FP64 inverse it applies) are staged in shared
      // memory with one bulk copy each, issued before anything else, where the launch has room
      const Real *rt = diag ? nullptr : (transposed ? g.tile(i, j) : g.tile(j, i));
      const double *xt = diag ? P.rinv + (size_t)i * nb * nb : (t.tgt ? P.rinv + (size_t)j * nb * nb : nullptr);
      const uint32_t rbytes = (uint32_t)(nb * nb * sizeof(Real)), xbytes = (uint32_t)(nb * nb * sizeof(double));
      unsigned char *stg = reinterpret_cast<unsigned char *>(sm) + kVecStageOff;
      const uint32_t room = ptx::dynamic_smem_bytes();
      const bool st_r = rt && aligned16(rt) && kVecStageOff + rbytes <= room;
      const uint32_t xoff = st_r ? rbytes : 0;
      const bool st_x = xt && aligned16(xt) && kVecStageOff + xoff + xbytes <= room;
      const Real *mr = st_r ? reinterpret_cast<const Real *>(stg) : rt;
      const double *mx = st_x ? reinterpret_cast<const double *>(stg + xoff) : xt;
      if ((st_r || st_x) && threadIdx.x == 0) {
        ptx::fence_proxy_async();
        ptx::mbar_arrive_expect_tx(&sh.bar, (st_r ? rbytes : 0) + (st_x ? xbytes : 0));
        if (st_r) ptx::bulk_g2s(stg, rt, rbytes, &sh.bar);
        if (st_x) ptx::bulk_g2s(stg + xoff, xt, xbytes, &sh.bar);
      }
      for (int k = tid; k < nb; k += NT) gs[k] = k < n_i ? __ldcg(gi + k) : 0.0;
      if (st_r || st_x) {  // bounded wait for the staged tiles
        if (!ptx::mbar_try_wait(&sh.bar, phase)) {
          const uint64_t t0 = ptx::globaltimer();
          while (!ptx::mbar_try_wait(&sh.bar, phase)) {
            if (ptx::globaltimer() - t0 > (uint64_t)p.timeout_ns) {
              sh.abort = 1;
              break;
            }
          }
        }
        phase ^= 1u;
      }
      __syncthreads();
      if (sh.abort) {
        if (tid == 0) set_error(p, HQR_ERR_TIMEOUT, -1);
        break;
      }
      // every thread owns one output and 1/H of its sum (no FP64 cross-lane reductions: a
      // warp-wide FP64 operation takes 16 cycles of the FP64 pipe)
      const int o = tid % nb, h = tid / nb, H = NT / nb;  // output index, part of the sum
      double acc = 0.0;
      if (o < n_out && h < H) {
        // out_o = sum_q M(row(q), col(q)) g_q: transposed M(q, o) (a column of M, o's own), else
        // M(o, q) (a row; consecutive threads read consecutive addresses). X is upper triangular.
        const int qlo = (diag && !transposed) ? o : 0;
        const int qhi = (diag && transposed) ? o + 1 : n_i;
        if (diag)
          acc = tile_dot(mx, nb, transposed, o, qlo + h, qhi, H, gs);
        else
          acc = tile_dot(mr, nb, transposed, o, qlo + h, qhi, H, gs);
      }
      if (h < H) part[h * nb + o] = acc;
      __syncthreads();
      if (tid < n_out) {
        double v = 0.0;
        for (int q = 0; q < H; ++q) v += part[q * nb + tid];
        v = diag ? v : __ldcg(go + tid) - v;
        if (!diag && t.tgt)
          gs[tid] = v;  // fused step: the inverse of tile j follows
        else
          go[tid] = v;
      }
      __syncthreads();
      if (!diag && t.tgt) {  // g_j <- X_j^T g_j (after TU) or X_j g_j (after U), X_j = R_jj^{-1}
        for (int k = tid; k < nb; k += NT)
          if (k >= n_out) gs[k] = 0.0;
        __syncthreads();
        acc = 0.0;
        if (o < n_out && h < H) {
          const int qlo = transposed ? 0 : o, qhi = transposed ? o + 1 : n_out;
          acc = tile_dot(mx, nb, transposed, o, qlo + h, qhi, H, gs);
        }
        if (h < H) part[h * nb + o] = acc;
        __syncthreads();
        if (tid < n_out) {
          double v = 0.0;
          for (int q = 0; q < H; ++q) v += part[q * nb + tid];
          go[tid] = v;
        }
        __syncthreads();
      }
      __syncthreads();
      break;
    }
    case OP_XUPD: {
      const int j = t.j, n_j = min(nb, P.N - j * nb);
      double md = 0.0, mx = 0.0;
      for (int c = tid; c < n_j; c += NT) {
        const double d = __ldcg(P.g + (size_t)j * nb + c);
        const double xn = __ldcg(P.x + (size_t)j * nb + c) + d;
        P.x[(size_t)j * nb + c] = xn;
        md = fma(d, d, md);
        mx = fma(xn, xn, mx);
      }
      if (tolm) {  // this tile's sum d^2 and sum x^2 (fixed order: threads, then warps)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          md += __shfl_xor_sync(0xffffffffu, md, o);
          mx += __shfl_xor_sync(0xffffffffu, mx, o);
        }
        if (lane == 0) {
          sm[warp] = md;
          sm[NWARP + warp] = mx;
        }
        __syncthreads();
        if (tid == 0) {
          for (int w = 1; w < NWARP; ++w) {
            md += sm[w];
            mx += sm[NWARP + w];
          }
          P.rn[2 * j] = md;
          P.rn[2 * j + 1] = mx;
        }
        __syncthreads();
      }
      break;
    }
    case OP_RCHK: {  // after every x update of round k: stop? compensate round k + 2?
      if (tid == 0) {
        RefineState *rs = P.rs;
        const int k = t.k;
        double sd = 0.0, sx = 0.0;
        for (int q = 0; q < g.n; ++q) {  // tile order: the same sum on every run
          sd += __ldcg(P.rn + 2 * q);
          sx += __ldcg(P.rn + 2 * q + 1);
        }
        const double c = sx > 0.0 ? sqrt(sd / sx) : (sd > 0.0 ? INFINITY : 0.0);
        rs->cval[k] = c;
        const int comp_k = __ldcg(&rs->mode[k]);
        const int comp_p = k >= 1 ? __ldcg(&rs->mode[k - 1]) : 0;
        const double cp = k >= 1 ? __ldcg(&rs->cval[k - 1]) : 0.0;
        if ((comp_k && c <= P.tol) || c == 0.0) {
          rs->met = 1;
          rs->conv = k + 1;
        } else if (comp_k && comp_p && !(c <= 0.9 * cp)) {
          rs->conv = k + 1;  // no more progress: the accuracy the low-precision R allows
          atomicCAS(P.status, 0, HQR_ERR_NOCONV);
        } else {
          // plain rounds until their corrections stop halving below 1e-6 (the plain residual's
          // floor) or reach the tolerance; from then on compensated residuals, which can
          // certify it
          if (k + 2 < P.maxit)
            rs->mode[k + 2] = (__ldcg(&rs->mode[k + 1]) || c <= P.tol || (c < 1e-6 && !(c <= 0.5 * cp))) ? 1 : 0;
          if (k == P.maxit - 1) atomicCAS(P.status, 0, HQR_ERR_NOCONV);
        }
      }
      break;
    }
    case OP_BTOG: {
      const int i = t.i, n_i = min(nb, P.N - i * nb);
      const Real *Bb = g.B + (size_t)i * nb * g.wb;
      for (int r = tid; r < n_i; r += NT) P.g[(size_t)i * nb + r] = (double)__ldcg(Bb + r);
      break;
    }
    case OP_PACK: {  // tile column j of the workspace, zero padded; column 0 also b and x = 0
      const int j = t.j, m = g.m;
      const long long per_col = (long long)m * nb * nb;
      Real *ws = g.A + (size_t)j * per_col;
      for (long long e = tid; e < per_col; e += NT) {
        const long long tile = e / ((long long)nb * nb);
        const int w = (int)(e - tile * nb * nb);
        const int cc = w / nb, rr = w - cc * nb;
        const int row = (int)tile * nb + rr, col = j * nb + cc;
        ws[e] = (row < P.M && col < P.N) ? A0[(long long)col * P.lda0 + row] : Real(0);
      }
      if (j == 0) {
        for (int r = tid; r < m * nb; r += NT) g.B[r] = r < P.M ? (Real)P.b[r] : Real(0);
        for (int c = tid; c < P.N; c += NT) P.x[c] = 0.0;
      }
      break;
    }
    case OP_RJOIN:  // a join of the round's residual rows: no work
    default:
      break;
  }
}

// ------------------------------------------------------------- scheduler --

__device__ __forceinline__ void push_ready(const EngineParams &p, int task) {
  const int qs = p.tasks[task].prio * kShards + task % kShards;
  const unsigned idx = atomicAdd(&p.ctl->tail[qs].v, 1u);
  ptx::st_release(&p.slots[(size_t)qs * shard_cap(p.ntasks) + idx], task + 1);
}

// Warp-wide claim on NQ priority classes x kShards ready rings (ring id =
// class * kShards + shard; within a class this CTA's home shard first).
// Each lane reads the head and tail of NQ / 4 rings at once, a ballot picks
// the highest-priority non-empty ring, and the lane that saw it claims that
// ring's head. All lanes return the ring (-1: every ring looked empty) and
// `pos`, the claimed position. Called by all 32 lanes of one warp.
template <int NQ>
__device__ __forceinline__ int warp_claim(CtlLine *head, const CtlLine *tail, unsigned &pos) {
  static_assert(NQ % 4 == 0 && kShards == 8, "a warp covers 4 classes x 8 shards per round");
  constexpr int G = NQ / 4;
  const int lane = threadIdx.x & 31;
  const int ring0 = (lane >> 3) * kShards + ((lane + (int)blockIdx.x) & (kShards - 1));
  while (true) {
    unsigned h[G], tl[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      h[g] = ptx::ld_relaxed_u32(&head[g * 32 + ring0].v);
      tl[g] = ptx::ld_relaxed_u32(&tail[g * 32 + ring0].v);
    }
    bool contended = false;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const unsigned m = __ballot_sync(0xffffffffu, h[g] < tl[g]);
      if (m == 0) continue;
      const int w = __ffs(m) - 1;
      int ok = 0;
      unsigned hh = h[g];
      if (lane == w) {
        while (hh < tl[g]) {
          const unsigned old = atomicCAS(&head[g * 32 + ring0].v, hh, hh + 1);
          if (old == hh) {
            ok = 1;
            break;
          }
          hh = old;
        }
      }
      if (__shfl_sync(0xffffffffu, ok, w)) {
        pos = __shfl_sync(0xffffffffu, hh, w);
        return g * 32 + __shfl_sync(0xffffffffu, ring0, w);
      }
      contended = true;  // another CTA took it: look again
      break;
    }
    if (!contended) return -1;
  }
}

// Wait (bounded) for the task id a pusher stores into a claimed ring slot.
// Returns the task, or -1 after setting HQR_ERR_TIMEOUT.
__device__ __forceinline__ int take_slot(const EngineParams &p, int *slot) {
  int v = ptx::ld_acquire(slot);
  const uint64_t t1 = ptx::globaltimer();
  while (v == 0) {
    if (ptx::globaltimer() - t1 > (uint64_t)p.timeout_ns) {
      set_error(p, HQR_ERR_TIMEOUT, -1);
      return -1;
    }
    __nanosleep(32);
    v = ptx::ld_acquire(slot);
  }
  __threadfence();
  return v - 1;
}

// Claim the next ready task (one warp, all lanes; the result in every lane).
// -1: finished or failed. `pending` (lane 0's) counts tasks this CTA
// completed but has not yet added to the global done counter; it is flushed
// whenever the queues look empty.
__device__ int pop_ready(const EngineParams &p, unsigned &pending) {
  const int lane = threadIdx.x & 31;
  const uint64_t t0 = ptx::globaltimer();
  const int cap = shard_cap(p.ntasks);
  unsigned sleep_ns = 32;
  while (true) {
    if (__shfl_sync(0xffffffffu, lane == 0 ? ptx::ld_relaxed((const int *)&p.ctl->status.v) : 0, 0) != 0) return -1;
    unsigned h = 0;
    const int qs = warp_claim<kNumQueues>(p.ctl->head, p.ctl->tail, h);
    if (qs >= 0) {
      int v = 0;
      if (lane == 0) v = take_slot(p, &p.slots[(size_t)qs * cap + h]);
      return __shfl_sync(0xffffffffu, v, 0);
    }
    int fin = 0;
    if (lane == 0) {
      if (pending) {
        __threadfence();
        atomicAdd(&p.ctl->done.v, pending);
        pending = 0;
      }
      if (ptx::ld_relaxed_u32(&p.ctl->done.v) >= (unsigned)p.ntasks) {
        fin = 1;
      } else if (ptx::globaltimer() - t0 > (uint64_t)p.timeout_ns) {
        set_error(p, HQR_ERR_TIMEOUT, -1);
        fin = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, fin, 0)) return -1;
    __nanosleep(sleep_ns);
    if (sleep_ns < 1024) sleep_ns *= 2;
  }
}

__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// Tensor memory and chunk barriers of a CTA of the tensor-core kernel
// variant (set up once per CTA, released at exit). Kernels that contain
// tcgen05 instructions run one CTA per SM, so that variant is separate and
// only launched for graphs with tensor-core problems.
template <bool TC>
__device__ __forceinline__ void tc_setup(tc::State &ts) {
  if constexpr (TC) {
    if (threadIdx.x == 0) {
      for (int c = 0; c < tc::NCH; ++c) {
        ptx::mbar_init(&ts.full[c], NT);
        ptx::mbar_init(&ts.img[c], 1);
      }
      ptx::mbar_init(&ts.done, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tc::tmem_alloc(&ts.tmem);
    tc::tc_fence_before();
  }
}

template <bool TC>
__device__ __forceinline__ void tc_release(tc::State &ts) {
  if constexpr (TC) {
    __syncthreads();
    tc::tc_fence_after();
    if (threadIdx.x < 32) tc::tmem_dealloc(ts.tmem);
  }
}

// A panel or update task of a tensor-core problem. Returns false on a timeout.
template <typename Real, bool TC>
__device__ bool tc_task(const EngineParams &p, const Geo<Real> &g, const Task &t, Shared<Real> &sh,
                        unsigned char *dyn, tc::State &ts, tc::Phases &tph) {
  if constexpr (TC && sizeof(Real) == 4) {
    if (t.op == OP_GEQRT || t.op == OP_TSQRT || t.op == OP_TTQRT) {
      const int mode = t.op == OP_GEQRT ? 1 : (t.op == OP_TSQRT ? 0 : 2);
      tc::panel(mode, g.tile(t.i, t.k), g.tile(t.r, t.k), g.tfac(mode == 1 ? 0 : 1, t.i, t.k), g.t32 != 0, dyn);
      return true;
    }
    const int mode = t.op == OP_UNMQR ? 1 : (t.op == OP_TSMQR ? 0 : 2);
    const bool pair = t.op != OP_UNMQR;
    return tc::update(mode, t.trans, g.tile(t.i, t.k), g.tfac(pair ? 1 : 0, t.i, t.k),
                      pair ? g.target(t, t.r) : nullptr, g.target(t, t.i), t.cw, dyn, ts, tph, &sh.abort,
                      p.timeout_ns);
  }
  return true;
}

template <typename Real, bool TC>
__global__ void __launch_bounds__(NT, TC ? 1 : 2) hqr_sched(EngineParams p) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  Real *dyn = reinterpret_cast<Real *>(dyn_raw);
  __shared__ Shared<Real> sh;
  __shared__ tc::State ts;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&sh.bar, 1);
    sh.abort = 0;
    sh.norelease = 0;
  }
  tc_setup<TC>(ts);
  __syncthreads();
  tc::tc_fence_after();
  uint32_t phase = 0;
  tc::Phases tph;
  // Warp 1 claims the CTA's next task while warp 0 releases the successors
  // of the last one. It also counts completed tasks (`pending`, flushed to
  // the global done counter whenever the queues look empty or 64 have
  // accumulated): a task counts as done once its results are written, before
  // its successors are released, which cannot end the run early since the
  // counter reaches the task count only when no task has unfinished
  // successors. Seven warps release the successors (a solve step has up to
  // one per tile of the vector). After a least-squares vector task, the most
  // critical successor that the release makes ready (successors are listed by
  // decreasing bottom level) stays with this CTA and runs next without a trip
  // through the queues: the solve chain pays neither the push nor another
  // CTA's claim per step (measured: 7.0 -> 4.3 us between steps), and the sum
  // of a column tile's A^T r partials, then the solve step that needs it, run as
  // soon as the last partial is done instead of queuing behind the other
  // columns' partials. After such a task warp 1 claims only if nothing was kept
  // (after the release), so a kept task never meets a claimed one. (Keeping
  // after factorization tasks as well cost the 512^2 FP64 latency case 2 %.)
  unsigned pending = 0;
  if (threadIdx.x == 0) {
    sh.kept = -1;
    sh.popped = -1;
  }
  if (threadIdx.x >= 32 && threadIdx.x < 64) {
    const int v = pop_ready(p, pending);
    if (threadIdx.x == 32) sh.task = v;
  }
  __syncthreads();
  while (true) {
    const int tid = sh.task;
    if (tid < 0) break;
    const Task t = p.tasks[tid];
    const Geo<Real> g(p.probs[t.pid]);
    const uint64_t t_start = (p.trace && threadIdx.x == 0) ? ptx::globaltimer() : 0;
    if (TC && t.op <= OP_TTMQR && p.probs[t.pid].tc) {
      if (!tc_task<Real, TC>(p, g, t, sh, dyn_raw, ts, tph) && threadIdx.x == 0) set_error(p, HQR_ERR_TIMEOUT, tid);
    } else if (t.op == OP_GEQRT || t.op == OP_TSQRT || t.op == OP_TTQRT)
      task_panel(p, g, t, sh, dyn, phase);
    else if (t.op <= OP_TTMQR)
      task_update(p, g, t, sh, dyn, phase);
    else
      task_vector<Real, TC ? 16 : 8>(p, p.probs[t.pid], g, t, reinterpret_cast<double *>(dyn_raw), sh, phase);
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    if (warp != 1) {  // warps 0, 2 .. 7 release the successors, warp 0 the most critical 32
      if (threadIdx.x == 0 && p.trace) {
        p.trace[3 * (size_t)tid + 0] = t_start;
        p.trace[3 * (size_t)tid + 1] = ptx::globaltimer();
        p.trace[3 * (size_t)tid + 2] = ((unsigned long long)blockIdx.x << 32) | smid();
      }
      ptx::fence_proxy_async();
      __threadfence();
      const int rw = warp == 0 ? 0 : warp - 1;  // release slot of this warp
      const int e_end = sh.norelease ? t.succ_begin : t.succ_end;
      const bool may_keep = warp == 0 && t.op >= OP_RESID;
      for (int e0 = t.succ_begin + 32 * rw; e0 < e_end; e0 += 32 * (NWARP - 1)) {
        const int e = e0 + (threadIdx.x & 31);
        int s = -1;
        bool ready = false;
        if (e < e_end) {
          s = p.succ[e];
          ready = atomicSub(&p.indeg[s], 1) == 1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ready);
        const int keeper = (e0 == t.succ_begin && may_keep && m) ? __ffs(m) - 1 : -1;
        if (ready) {
          if ((int)(threadIdx.x & 31) == keeper)
            *(volatile int *)&sh.kept = s;
          else
            push_ready(p, s);
        }
      }
      __syncwarp();
      // a kept task's other predecessors published their results before their own decrements
      // (fence, then atomic): this fence orders its reads after the decrement that made it ready,
      // as take_slot does for a claimed task
      __threadfence();
    } else {  // warp 1 claims the next task meanwhile
      if (threadIdx.x == 32 && ++pending >= 64) {
        __threadfence();
        atomicAdd(&p.ctl->done.v, pending);
        pending = 0;
      }
      // after a vector task the claim waits for the release (a successor may be kept)
      const int v = (sh.abort || t.op >= OP_RESID) ? -1 : pop_ready(p, pending);
      if (threadIdx.x == 32) sh.popped = v;
    }
    __syncthreads();
    if (t.op >= OP_RESID && sh.kept < 0 && !sh.abort && warp == 1) {  // nothing kept: claim now
      const int v = pop_ready(p, pending);
      if (threadIdx.x == 32) sh.popped = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the next task: the kept one, else the claimed one
      sh.task = sh.kept >= 0 ? sh.kept : sh.popped;
      sh.kept = -1;
      sh.popped = -1;
      sh.norelease = 0;
    }
    __syncthreads();
    if (sh.abort) break;
  }
  // a bulk copy that outlived its wait must land before the CTA exits
  if (sh.abort && threadIdx.x == 0) {
    const uint64_t t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(&sh.bar, phase) && ptx::globaltimer() - t0 < 1000000000ull) {
    }
  }
  tc_release<TC>(ts);
}


// ------------------------------------------------------------ server mode --
// A resident variant of the scheduler for continuous batching: requests
// (each a least-squares task graph in a pool range, with its own problem
// slot) arrive through an inbox written by the host while the kernel runs.
// A CTA with nothing to do claims the next inbox entry and releases the
// request's initial tasks; when a request's last task completes, its
// sequence number is written to host-mapped memory. Ready queues are rings
// (slots cleared after use). The kernel exits once the host has set `stop`
// and no task is outstanding.

// Server ready rings: kAgeClasses request-age classes x kNumQueues
// critical-path classes x kShards. The age class of a request is its rank
// among the requests not yet finished, in admission order (0-1: 0, 2-7: 1,
// 8-31: 2, else 3), taken when a task is released: the oldest requests
// run first and newer ones fill the CTAs they leave idle, so that requests
// complete roughly in arrival order under overload instead of all sharing
// the GPU until the end.
constexpr int kAgeClasses = 4;
constexpr int kServeQueues = kAgeClasses * kNumQueues;

struct ServeCtl {
  CtlLine inbox_head, inbox_tail, stop, outstanding, finished;
  CtlLine head[kServeQueues * kShards];
  CtlLine tail[kServeQueues * kShards];
};

struct InboxEntry {
  int slot, task_base, ninit, ntasks;
};

struct ServeParams {
  EngineParams e;                 // probs (per slot), task / successor / in-degree pools, rings, status
  ServeCtl *sc;
  const InboxEntry *inbox;
  int inbox_cap;                  // power of two
  const int *initlist;            // initial ready tasks of a request at [task_base, task_base + ninit)
  int *req_done;                  // per slot: tasks completed
  const int *req_total;           // per slot: tasks of the request
  const long long *req_seq;       // per slot: sequence number of the request
  volatile long long *comp;       // host-mapped, per slot: last completed sequence number
  int ring_cap;                   // power of two, per queue shard
};

__device__ __forceinline__ long long ld_acquire_sys_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// A pool task, read around L1 (pool entries are rewritten for every request).
__device__ __forceinline__ Task load_task_cg(const Task *tp) {
  static_assert(sizeof(Task) == 40, "Task is read in 8-byte pieces");
  Task t;
  const int2 *src = reinterpret_cast<const int2 *>(tp);
  int2 *dst = reinterpret_cast<int2 *>(&t);
#pragma unroll
  for (int q = 0; q < 5; ++q) dst[q] = __ldcg(src + q);
  return t;
}

// Rank estimate: requests admitted before this one minus requests finished
// (negative when later requests finished first: the oldest class then).
__device__ __forceinline__ int age_class(const ServeParams &sp, int slot) {
  const int rank = (int)((unsigned)(__ldcg(sp.req_seq + slot) - 1) - ptx::ld_relaxed_u32(&sp.sc->finished.v));
  return rank < 2 ? 0 : rank < 8 ? 1 : rank < 32 ? 2 : 3;
}

__device__ __forceinline__ void serve_push(const ServeParams &sp, int task, int age) {
  const int2 head = __ldcg(reinterpret_cast<const int2 *>(sp.e.tasks + task));
  const int prio = (int)(signed char)((head.x >> 8) & 0xff);  // byte 1 of the task record
  const int qs = (age * kNumQueues + prio) * kShards + task % kShards;
  const unsigned idx = atomicAdd(&sp.sc->tail[qs].v, 1u);
  ptx::st_release(&sp.e.slots[(size_t)qs * sp.ring_cap + (idx & (unsigned)(sp.ring_cap - 1))], task + 1);
}

// Besides -1 (stop, error) a CTA also leaves after kIdleExitNs without any
// work, so that an unused server never holds the GPU; the host relaunches
// the kernel when new work arrives.
constexpr uint64_t kIdleExitNs = 1000000000ull;

// Claim the next ready task or inbox entry (warp 0, all lanes; the task in
// every lane, -1 to leave).
__device__ int serve_pop(const ServeParams &sp, unsigned &pending) {
  const EngineParams &p = sp.e;
  const int lane = threadIdx.x & 31;
  unsigned sleep_ns = 64;
  const uint64_t idle_since = ptx::globaltimer();
  unsigned seen_out = 0xffffffffu;  // watchdog: outstanding count last seen and since when
  uint64_t seen_at = idle_since;
  while (true) {
    if (__shfl_sync(0xffffffffu, lane == 0 ? ptx::ld_relaxed((const int *)&p.ctl->status.v) : 0, 0) != 0) return -1;
    unsigned h = 0;
    const int qs = warp_claim<kServeQueues>(sp.sc->head, sp.sc->tail, h);
    if (qs >= 0) {
      int v = 0;
      if (lane == 0) {
        int *slot = &p.slots[(size_t)qs * sp.ring_cap + (h & (unsigned)(sp.ring_cap - 1))];
        v = take_slot(p, slot);
        if (v >= 0) {
          *slot = 0;  // the ring slot can be reused
          __threadfence();
        }
      }
      return __shfl_sync(0xffffffffu, v, 0);
    }
    // new request? (lane 0 claims the entry, the warp releases its initial tasks)
    int base = 0, ninit = -1, age = 0;
    if (lane == 0) {
      const unsigned ih = ptx::ld_relaxed_u32(&sp.sc->inbox_head.v);
      if (ih < (unsigned)ld_acquire_sys_u32(&sp.sc->inbox_tail.v)) {
        ninit = 0;
        if (atomicCAS(&sp.sc->inbox_head.v, ih, ih + 1) == ih) {
          const InboxEntry *en = sp.inbox + (ih & (unsigned)(sp.inbox_cap - 1));
          const int nt = __ldcg(&en->ntasks);
          base = __ldcg(&en->task_base);
          ninit = __ldcg(&en->ninit);
          age = age_class(sp, __ldcg(&en->slot));
          atomicAdd(&sp.sc->outstanding.v, (unsigned)nt);
        }
      }
    }
    ninit = __shfl_sync(0xffffffffu, ninit, 0);
    if (ninit >= 0) {
      base = __shfl_sync(0xffffffffu, base, 0);
      age = __shfl_sync(0xffffffffu, age, 0);
      for (int k = lane; k < ninit; k += 32) serve_push(sp, __ldcg(sp.initlist + base + k), age);
      continue;
    }
    int leave = 0;
    if (lane == 0) {
      if (pending) {
        __threadfence();
        atomicSub(&sp.sc->outstanding.v, pending);
        pending = 0;
      }
      const unsigned outst = ptx::ld_relaxed_u32(&sp.sc->outstanding.v);
      const uint64_t now = ptx::globaltimer();
      if (outst != seen_out) {
        seen_out = outst;
        seen_at = now;
      }
      if (outst == 0 && ld_acquire_sys_u32(&sp.sc->stop.v) != 0 &&
          ptx::ld_relaxed_u32(&sp.sc->inbox_head.v) == (unsigned)ld_acquire_sys_u32(&sp.sc->inbox_tail.v)) {
        leave = 1;
      } else if (outst != 0) {  // work outstanding but no task finished for the whole limit: a lost dependency
        if (now - seen_at > (uint64_t)p.timeout_ns) {
          set_error(p, HQR_ERR_TIMEOUT, -1);
          leave = 1;
        }
      } else if (now - idle_since > kIdleExitNs) {
        leave = 1;  // idle: leave; the host relaunches on new work
      }
    }
    if (__shfl_sync(0xffffffffu, leave, 0)) return -1;
    __nanosleep(sleep_ns);
    if (sleep_ns < 4096) sleep_ns *= 2;
  }
}

template <typename Real, bool TC>
__global__ void __launch_bounds__(NT, TC ? 1 : 2) hqr_serve(ServeParams sp) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  Real *dyn = reinterpret_cast<Real *>(dyn_raw);
  __shared__ Shared<Real> sh;
  __shared__ tc::State ts;
  const EngineParams &p = sp.e;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&sh.bar, 1);
    sh.abort = 0;
    sh.norelease = 0;
  }
  tc_setup<TC>(ts);
  __syncthreads();
  tc::tc_fence_after();
  uint32_t phase = 0;
  tc::Phases tph;
  unsigned pending = 0;
  while (true) {
    if (threadIdx.x < 32) {
      const int v = serve_pop(sp, pending);
      if (threadIdx.x == 0) sh.task = v;
    }
    __syncthreads();
    const int tid = sh.task;
    if (tid < 0) break;
    const Task t = load_task_cg(p.tasks + tid);
    Problem P;
    {
      const int4 *src = reinterpret_cast<const int4 *>(p.probs + t.pid);
      int4 *dst = reinterpret_cast<int4 *>(&P);
      for (int q = 0; q < (int)(sizeof(Problem) / 16); ++q) dst[q] = __ldcg(src + q);
    }
    const Geo<Real> g(P);
    if (TC && t.op <= OP_TTMQR && P.tc) {
      if (!tc_task<Real, TC>(p, g, t, sh, dyn_raw, ts, tph) && threadIdx.x == 0) set_error(p, HQR_ERR_TIMEOUT, tid);
    } else if (t.op == OP_GEQRT || t.op == OP_TSQRT || t.op == OP_TTQRT)
      task_panel(p, g, t, sh, dyn, phase);
    else if (t.op <= OP_TTMQR)
      task_update(p, g, t, sh, dyn, phase);
    else
      task_vector<Real, TC ? 16 : 8>(p, P, g, t, reinterpret_cast<double *>(dyn_raw), sh, phase);
    __syncthreads();
    if (threadIdx.x < 32) {  // warp 0 releases the successors, 32 at a time
      ptx::fence_proxy_async();
      __threadfence();
      if (t.succ_end > t.succ_begin) {
        const int age = __shfl_sync(0xffffffffu, threadIdx.x == 0 ? age_class(sp, t.pid) : 0, 0);
        for (int e = t.succ_begin + (int)threadIdx.x; e < t.succ_end; e += 32) {
          const int s = __ldcg(p.succ + e);
          if (atomicSub(&p.indeg[s], 1) == 1) serve_push(sp, s, age);
        }
      }
    }
    if (threadIdx.x == 0) {
      if (atomicAdd(&sp.req_done[t.pid], 1) + 1 == __ldcg(sp.req_total + t.pid)) {
        __threadfence_system();
        sp.comp[t.pid] = __ldcg(sp.req_seq + t.pid);
        __threadfence_system();
        atomicAdd(&sp.sc->finished.v, 1u);  // later requests move up an age rank
      }
      if (++pending >= 32) {  // keep the outstanding count current for the watchdogs
        __threadfence();
        atomicSub(&sp.sc->outstanding.v, pending);
        pending = 0;
      }
    }
    if (sh.abort) break;
  }
  if (sh.abort && threadIdx.x == 0) {
    const uint64_t t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(&sh.bar, phase) && ptx::globaltimer() - t0 < 1000000000ull) {
    }
  }
  tc_release<TC>(ts);
}

// Shared memory (bytes) of the scheduler kernel for tensor-core problems.
inline size_t engine_smem_bytes_tc() {
  const size_t vec = (size_t)(2 * NT + 256) * sizeof(double);
  return std::max<size_t>({(size_t)tc::SMEM_BYTES, (size_t)tc::PANEL_SMEM, vec});
}

// Shared memory (bytes) of the scheduler kernel for a problem configuration.
template <typename Real>
__host__ __device__ inline size_t engine_smem_bytes(int nb, int ib, int w, int wt, int vc) {
  const int lds = nb + smem_pad<Real>(), ldt = ib + smem_pad<Real>();
  // scratch: FP32 GEMMs keep up to 4 K-groups of partial output blocks
  const size_t fac = sizeof(Real) == 4 ? 4 : 1;
  const size_t su = fac * (((vc + 3) / 4) * ((w + 3) / 4) * 16);
  const size_t scr_u = su > (size_t)NT ? su : (size_t)NT;
  const size_t sp1 = fac * (((ib + 3) / 4) * ((wt + 3) / 4) * 16), sp2 = fac * (((ib + 3) / 4) * ((ib + 3) / 4) * 16);
  const size_t sp = sp1 > sp2 ? sp1 : sp2;
  const size_t scr_p = sp > (size_t)NT ? sp : (size_t)NT;
  const int ldq = sizeof(Real) == 8 ? ldt : ib;  // T of a block
  const size_t upd = (size_t)lds * (2 * w + vc) + (size_t)ib * ldq + (size_t)ib * w + scr_u;
  const size_t cbg = (size_t)(lds * wt > ib * ib ? lds * wt : ib * ib);
  const size_t pan = (size_t)lds * ib + (size_t)ldt * (ib + wt) + (size_t)ib * ldq + cbg +
                     (size_t)ib * wt + scr_p;
  const size_t vec = (size_t)(2 * NT + 256) * sizeof(double);  // FP64 vector tasks
  const size_t tiles = sizeof(Real) * (upd > pan ? upd : pan);
  return tiles > vec ? tiles : vec;
}

}  // namespace hqr
