// Tensor-core (tcgen05) tile kernels of the FP32 path, tile size 128.
//
// Updates (UNMQR / TSMQR / TTMQR, Alg. 2) of a whole tile column (or of a
// right-hand-side block) with the full 128 x 128 compact-WY factor T of the
// panel tile, as products with M = 128 on the 5th-generation tensor cores:
//   Q^T C = C - V T^T V^T C:  W = V^T C_b (+ C_t for TS/TT, whose V has an
//     identity top block); C_t -= T^T W (TS/TT); C_b -= Y W, Y = V T^T
//     precomputed by the panel task, so both updates come from the same W;
//   Q C = C - V T V^T C:  W = V^T C_b (+ C_t); W' = T W; C_t -= W';
//     C_b -= V W' (only factorizations that keep V and T apply Q).
// Each product runs as kind::f16 MMAs on BF16 operands split three ways
// ("BF16x3": x = b0 + b1 + b2 with b0 = bf16(x), b1 = bf16(x - b0), b2 =
// bf16(x - b0 - b1), all rounded to nearest, |x - b0 - b1 - b2| <= 2^-27 |x|)
// and six products per K step (b0 b0' + b0 b1' + b1 b0' + b0 b2' + b1 b1' +
// b2 b0'; the dropped terms are below 2^-26 of |x x'|), accumulating in FP32
// in tensor memory (one accumulator per K chunk of 32, summed in FP32 in the
// epilogue). The updates thus keep FP32 accuracy, which the
// corrected semi-normal-equation refinement needs, at the tensor-core cost
// of three tf32 products. With N = 128 columns per task an MMA runs at the
// pipe's full rate (N <= 64 costs the same time per instruction).
//
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: core matrices of 8 rows x 16 bytes (8 bf16), element (row, k) at
//   (row & 7) * 16 + (row >> 3) * SBO + (k & 7) * 2 + (k >> 3) * LBO.
// A product streams its operands in 4 chunks of K = 32, each in its own
// shared-memory stage; every thread loads its pieces of a chunk two chunks
// ahead into registers (L2-only loads, so no stale L1 lines across tasks).
// The operand images of the panel (V^T, T^T, Y, and V for Q) arrive by one
// bulk copy per chunk; the next image is requested while the epilogue of the
// previous product runs. The intermediate W^T is resident (K = 128) with
// LBO = 144 bytes so that its transposed writes from tensor memory are free
// of bank conflicts. The C tiles stay in global memory: the threads split
// C_b^T into the stages from there, and the epilogues read and write C with
// a warp's lanes on consecutive rows. Hand-off uses mbarriers: every thread
// arrives on a chunk's barrier after writing it, one thread issues that
// chunk's MMAs, and one commit signals the end of a product. Every wait is
// bounded by the global timer.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "ptx.cuh"

namespace hqr {
namespace tc {

constexpr int NB = 128;          // tile size of the tensor-core path
constexpr int WMAX = 128;        // widest column slab of an update task (a whole tile)
constexpr int KC = 32;           // K extent of one chunk (two MMA K steps of 16)
constexpr int NCH = NB / KC;     // chunks per product (each in its own stage)
constexpr int DT = 2;            // chunks loaded ahead in registers
constexpr int NP = 3;            // BF16 pieces of an FP32 value
constexpr int KS_ACC = 2;                  // MMA K steps (of 16) chained in one accumulator
constexpr int NACC = NCH * (KC / 16) / KS_ACC;  // accumulators: one per K chunk of 32
constexpr int TMEM_COLS = NACC * WMAX;  // 512 columns: one product's accumulators (all of the SM's)
constexpr int NTHR = 256;

constexpr uint32_t LBO_C = 128, SBO_C = (KC / 8) * 128;      // chunk buffers: 8-row groups of 512 B
constexpr uint32_t A_PC = (NB / 8) * SBO_C;                  // one piece of a 128 x 32 chunk: 8192 B
constexpr uint32_t B_PC = (WMAX / 8) * SBO_C;                // one piece of a 128 x 32 chunk: 8192 B
constexpr uint32_t LBO_W = 144, SBO_W = (NB / 8) * LBO_W;    // resident W^T (K = 128)
constexpr uint32_t W_PC = (WMAX / 8) * SBO_W;                // one piece: 36864 B
constexpr uint32_t OFF_W = 0;
constexpr uint32_t STAGE_A = NP * (A_PC + B_PC);             // product A stage: A pieces, B pieces
constexpr uint32_t STAGE_BC = NP * A_PC;                     // products B, C: A pieces
constexpr uint32_t OFF_RING_A = 0;                           // product A: W region is free
constexpr uint32_t OFF_RING_BC = NP * W_PC;
constexpr uint32_t SMEM_A = OFF_RING_A + NCH * STAGE_A;      // 196608
constexpr uint32_t SMEM_BC = OFF_RING_BC + NCH * STAGE_BC;   // 208896
constexpr uint32_t SMEM_BYTES = SMEM_A > SMEM_BC ? SMEM_A : SMEM_BC;  // 208896 (the C tiles stay in global memory)

// Per panel tile (i, k, GEQRT or kill) the panel task stores a "T record":
// the update operands already split into BF16 pieces in the chunk layout of
// the shared-memory stages (chunk c: pieces 0, 1, 2 of 128 x 32 elements),
// so that an update stages each chunk with one bulk copy: T^T (reflector,
// reflector'), V^T (reflector, row) and Y = V T^T (row, reflector), with V
// masked to its structure (unit lower, upper, full); then, for
// factorizations that keep them (apply Q, read T), V (row, reflector) and the
// FP32 factor T (128 x 128, column-major, zeros below the diagonal).
// Least-squares problems only apply Q^T and leave those two out.
constexpr uint32_t IMG_BYTES = NCH * NP * A_PC;                  // 98304
constexpr uint32_t REC_TB = 0;                                   // byte offsets in a record
constexpr uint32_t REC_VA = REC_TB + IMG_BYTES;
constexpr uint32_t REC_Y = REC_VA + IMG_BYTES;
constexpr uint32_t REC_VC = REC_Y + IMG_BYTES;
constexpr uint32_t REC_T32 = REC_VC + IMG_BYTES;
constexpr uint32_t T_RECORD_IMG = REC_VC / 4;                    // floats per record without V and T: 73728
constexpr uint32_t T_RECORD = (REC_T32 + NB * NB * 4) / 4;       // with them: 114688

// Per-CTA state of the tensor path (in the kernel's static shared memory).
struct State {
  uint64_t full[NCH];   // chunk c staged by every thread
  uint64_t img[NCH];    // chunk c of an operand image arrived (bulk copy)
  uint64_t done;        // every MMA of a product completed
  uint32_t tmem;
  int pad;
};

// ------------------------------------------------------------------- PTX --

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t *dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ptx::smem_addr(dst)),
               "r"((uint32_t)TMEM_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"((uint32_t)TMEM_COLS)
               : "memory");
}

// Shared-memory matrix descriptor: start, LBO, SBO (all bytes, 16-aligned),
// no swizzle, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   ptx::smem_addr(bar))
               : "memory");
}

// 32 lanes x 16 columns of 32 bits: this thread gets lane (base + laneid),
// columns col .. col + 15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float4 ldcg4(const float *p) { return __ldcg(reinterpret_cast<const float4 *>(p)); }

// x = b0 + b1 + b2 + e, |e| <= 2^-27 |x| (bf16 keeps FP32's exponent range;
// each difference is exact in FP32). Returns the three pieces' bit patterns.
__device__ __forceinline__ void split3(float x, uint32_t &p0, uint32_t &p1, uint32_t &p2) {
  const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
  p0 = __bfloat16_as_ushort(b0);
  p1 = __bfloat16_as_ushort(b1);
  p2 = __bfloat16_as_ushort(b2);
}


// ------------------------------------------------------------- pipeline --

// Bounded wait on an mbarrier phase. Returns false (and sets *abort) when the
// limit passes or another thread already gave up.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort, long long limit_ns) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ptx::globaltimer();
  while (!ptx::mbar_try_wait(bar, parity)) {
    if (*abort || ptx::globaltimer() - t0 > (uint64_t)limit_ns) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// Parity of the chunk barriers (all flip once per product) and of the done
// barrier, tracked identically by every thread.
struct Phases {
  uint32_t full = 0, img = 0, done = 0;
};

// Element masks of the reflector block V at (row, reflector):
//  0 none (TS: full tile), 1 unit lower (GE), 2 upper incl. diagonal (TT).
__device__ __forceinline__ float vmask(int mode, int row, int refl, float x) {
  if (mode == 1) return row > refl ? x : (row == refl ? 1.f : 0.f);
  if (mode == 2) return row <= refl ? x : 0.f;
  return x;
}

// Source of a streamed operand. Element (m, k):
//  natural:    p[m * ld + k]   (k contiguous: two 16-byte loads per piece)
//  transposed: p[k * ld + m]   (m contiguous: eight coalesced 4-byte loads)
struct Src {
  const float *p;
  int ld;
  int transposed;
  int rows;     // valid rows (m < rows); others are zero
  int vmode;    // vmask mode, with (row, refl) = natural ? (k, m) : (m, k); -1: none
  int shared;   // p points to shared memory (a staged slab): plain loads
};

// A piece: row m, k group kg (k = 8 kg .. 8 kg + 7 of the chunk), 8 floats.
struct Piece {
  float4 lo4, hi4;
};

// Piece u of this thread in a chunk of `rows` rows (rows * 4 pieces). Natural
// operands: eight lanes take eight consecutive rows of one k group (a
// 128-byte shared-memory row per quarter warp; each row's 128 global bytes
// by four lanes); transposed ones: lanes take consecutive rows.
__device__ __forceinline__ void piece_coords(const Src &s, int rows, int u, int &m, int &kg) {
  const int p = threadIdx.x + NTHR * u;
  if (!s.transposed) {
    m = (p >> 5) * 8 + (p & 7);
    kg = (p >> 3) & 3;
    if (rows < NB) m = ((p >> 5) % (rows / 8)) * 8 + (p & 7);
  } else {
    m = p % rows;
    kg = p / rows;
  }
}

__device__ __forceinline__ Piece load_piece(const Src &s, int c, int m, int kg) {
  Piece r;
  const int k0 = c * KC + kg * 8;
  if (m >= s.rows) {
    r.lo4 = r.hi4 = make_float4(0.f, 0.f, 0.f, 0.f);
  } else if (!s.transposed) {
    const float *q = s.p + (size_t)m * s.ld + k0;
    if (s.shared) {
      r.lo4 = *reinterpret_cast<const float4 *>(q);
      r.hi4 = *reinterpret_cast<const float4 *>(q + 4);
    } else {
      r.lo4 = ldcg4(q);
      r.hi4 = ldcg4(q + 4);
    }
  } else {
    const float *q = s.p + (size_t)k0 * s.ld + m;
    r.lo4.x = __ldcg(q);
    r.lo4.y = __ldcg(q + s.ld);
    r.lo4.z = __ldcg(q + 2 * (size_t)s.ld);
    r.lo4.w = __ldcg(q + 3 * (size_t)s.ld);
    r.hi4.x = __ldcg(q + 4 * (size_t)s.ld);
    r.hi4.y = __ldcg(q + 5 * (size_t)s.ld);
    r.hi4.z = __ldcg(q + 6 * (size_t)s.ld);
    r.hi4.w = __ldcg(q + 7 * (size_t)s.ld);
  }
  return r;
}

// Mask, split and store a piece: three 16-byte stores (one per BF16 piece).
__device__ __forceinline__ void store_piece(const Src &s, const Piece &x, int c, int m, int kg, unsigned char *buf,
                                            uint32_t piece_bytes) {
  float v[8] = {x.lo4.x, x.lo4.y, x.lo4.z, x.lo4.w, x.hi4.x, x.hi4.y, x.hi4.z, x.hi4.w};
  if (s.vmode >= 0) {
    const int k0 = c * KC + kg * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      v[e] = s.transposed ? vmask(s.vmode, m, k0 + e, v[e]) : vmask(s.vmode, k0 + e, m, v[e]);
  }
  uint32_t w[NP][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    uint32_t a0, a1, a2, b0, b1, b2;
    split3(v[e], a0, a1, a2);
    split3(v[e + 1], b0, b1, b2);
    w[0][e / 2] = a0 | (b0 << 16);
    w[1][e / 2] = a1 | (b1 << 16);
    w[2][e / 2] = a2 | (b2 << 16);
  }
  const uint32_t off = (uint32_t)(m & 7) * 16 + (uint32_t)(m >> 3) * SBO_C + (uint32_t)kg * LBO_C;
#pragma unroll
  for (int q = 0; q < NP; ++q)
    *reinterpret_cast<uint4 *>(buf + q * piece_bytes + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// Registers of a product's streamed operands: A, DT chunks ahead (2 pieces
// per thread and chunk), and B (product A only: all NCH chunks, requested at
// task start so that a single L2 round trip precedes the MMAs).
struct Fetch {
  Piece a[DT][2];
  Piece b[NCH][2];
};

__device__ __forceinline__ void fetch_a(const Src &s, int c, Piece (&r)[2]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int m, kg;
    piece_coords(s, NB, u, m, kg);
    r[u] = load_piece(s, c, m, kg);
  }
}

__device__ __forceinline__ void fetch_b(const Src &s, int c, Piece (&r)[2]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int m, kg;
    piece_coords(s, WMAX, u, m, kg);
    r[u] = load_piece(s, c, m, kg);
  }
}

// The six BF16 products of one K step, small terms first, accumulating.
__device__ __forceinline__ void issue_kstep(uint32_t tmem, uint32_t idesc, uint32_t a, uint32_t apb, uint32_t b,
                                            uint32_t bpb, uint32_t blbo, uint32_t bsbo, bool first) {
  const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const uint64_t ad = sdesc(a + (uint32_t)pa[t] * apb, LBO_C, SBO_C);
    const uint64_t bd = sdesc(b + (uint32_t)pb[t] * bpb, blbo, bsbo);
    mma_bf16(tmem, ad, bd, idesc, (first && t == 0) ? 0u : 1u);
  }
}

// D[128 x n] = A B^T over K = 128. A is either an operand image in global
// memory (`img`: one bulk copy per chunk, issued at once by one thread,
// possibly already by the caller) or gathered by every thread from `sa`
// (its first DT chunks already in `f`) and split into BF16 pieces; B is
// streamed from `sb` (product A: the staged C_b slab, split by the threads)
// or read from the resident W^T buffer (sb == nullptr). The first DT chunks
// of the next product's gathered operand `next` (if any) are requested into
// free registers: at once when A is an image, else while the last chunks are
// consumed. One thread issues each chunk's MMAs once its pieces are in
// place. Returns false on a timeout (the CTA's abort flag is set).
// The bulk copies of an operand image into a product's stages (one thread).
__device__ __forceinline__ void issue_image(const unsigned char *img, unsigned char *smem, uint32_t ring,
                                            uint32_t stage_bytes, State &st) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    ptx::mbar_arrive_expect_tx(&st.img[c], NP * A_PC);
    ptx::bulk_g2s(smem + ring + (uint32_t)c * stage_bytes, img + (size_t)c * NP * A_PC, NP * A_PC, &st.img[c]);
  }
}

__device__ bool product(const Src &sa, const unsigned char *img, const Src *sb, const Src *next, Fetch &f,
                        unsigned char *smem, State &st, Phases &ph, uint32_t tmem, int n, volatile int *abort,
                        long long limit_ns, bool img_issued = false, bool wait = true) {
  const int tid = threadIdx.x;
  const bool streamB = sb != nullptr, useImg = img != nullptr;
  const bool threadsWrite = !useImg || streamB;  // chunk hand-off through the "full" barriers
  const uint32_t ring = streamB ? OFF_RING_A : OFF_RING_BC;
  const uint32_t stage_bytes = streamB ? STAGE_A : STAGE_BC;
  const uint32_t idesc = idesc_bf16(n);
  const uint32_t sbase = ptx::smem_addr(smem);
  if (useImg && !img_issued && tid == 0) issue_image(img, smem, ring, stage_bytes, st);
  if (useImg && next)
#pragma unroll
    for (int c = 0; c < DT; ++c) fetch_a(*next, c, f.a[c]);
  bool ok = true;
  const uint32_t pf = ph.full & 1u, pi = ph.img & 1u;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    unsigned char *stage = smem + ring + (uint32_t)c * stage_bytes;
    const int slot = c % DT;
    if (!useImg) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        int m, kg;
        piece_coords(sa, NB, u, m, kg);
        store_piece(sa, f.a[slot][u], c, m, kg, stage, A_PC);
      }
    }
    if (streamB) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        int m, kg;
        piece_coords(*sb, WMAX, u, m, kg);
        store_piece(*sb, f.b[c][u], c, m, kg, stage + NP * A_PC, B_PC);
      }
    }
    if (c + DT < NCH) {
      if (!useImg) fetch_a(sa, c + DT, f.a[slot]);
    } else if (next && !useImg) {
      fetch_a(*next, c + DT - NCH, f.a[slot]);
    }
    if (threadsWrite) {
      fence_async_smem();
      mbar_arrive(&st.full[c]);
    }
    if (tid == 0) {
      if (useImg && !wait_bar(&st.img[c], pi, abort, limit_ns)) ok = false;
      if (threadsWrite && !wait_bar(&st.full[c], pf, abort, limit_ns)) ok = false;
      tc_fence_after();
      if (ok) {
        const uint32_t a = sbase + ring + (uint32_t)c * stage_bytes;
#pragma unroll
        for (int ks = 0; ks < KC / 16; ++ks) {
          const int acc = (c * (KC / 16) + ks) / KS_ACC;  // this K step's accumulator
          const bool first = (c * (KC / 16) + ks) % KS_ACC == 0;
          const uint32_t dk = tmem + (uint32_t)acc * WMAX;
          const uint32_t ak = a + (uint32_t)ks * 2 * LBO_C;
          if (streamB)
            issue_kstep(dk, idesc, ak, A_PC, a + NP * A_PC + (uint32_t)ks * 2 * LBO_C, B_PC, LBO_C, SBO_C, first);
          else
            issue_kstep(dk, idesc, ak, A_PC, sbase + OFF_W + (uint32_t)(c * KC / 8 + ks * 2) * LBO_W, W_PC,
                        LBO_W, SBO_W, first);
        }
      }
    }
  }
  if (threadsWrite) ph.full ^= 1u;
  if (useImg) ph.img ^= 1u;
  if (tid == 0) mma_commit(&st.done);
  if (!wait) return ok && !*abort;
  if (!wait_bar(&st.done, ph.done & 1u, abort, limit_ns)) ok = false;
  ph.done ^= 1u;
  tc_fence_after();
  return ok && !*abort;
}

// Completion of a product issued with wait = false (every thread).
__device__ __forceinline__ bool product_wait(State &st, Phases &ph, volatile int *abort, long long limit_ns) {
  const bool ok = wait_bar(&st.done, ph.done & 1u, abort, limit_ns);
  ph.done ^= 1u;
  tc_fence_after();
  return ok && !*abort;
}

// Sum of the K-chunk accumulators (columns col, col + 64, ...) of 16
// columns, in K order with round-to-nearest FP32 additions: each
// accumulator takes the MMAs of KS_ACC K steps only, which keeps the
// accumulation error of the tensor cores over a short chain.
__device__ __forceinline__ void tmem_sum16(uint32_t taddr, float (&v)[16]) {
  float w[NACC][16];
#pragma unroll
  for (int c = 0; c < NACC; ++c) tmem_ld16(taddr + (uint32_t)c * WMAX, w[c]);
  tmem_wait_ld();
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    float x = w[0][q];
#pragma unroll
    for (int c = 1; c < NACC; ++c) x += w[c][q];
    v[q] = x;
  }
}

// Accumulator elements of this thread in the epilogues: row m = 32 (warp &
// 3) + laneid (the tensor-memory lanes its warp may read), columns 16 g ..
// 16 g + 15 for the column groups g = (warp >> 2) + 2 e, e = 0 .. 3 (n <= 128).
// The C tiles stay in global memory (column col at col * 128 floats): a warp's
// accesses to one column are 128 consecutive bytes. A thread's 64 elements of
// a C tile in this layout ("C registers") are loaded ahead of the epilogue
// that needs them, while the tensor cores run the product before it.
typedef float CRegs[4][16];

__device__ __forceinline__ void load_c(const float *c, int cw, CRegs &r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = 32 * (warp & 3) + lane;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int g = (warp >> 2) + 2 * e;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = 16 * g + q;
      r[e][q] = (c && col < cw) ? __ldcg(c + (size_t)col * NB + m) : 0.f;
    }
  }
}

// Offset of element (n = column, k = reflector) in a piece of the resident
// W^T buffer.
__device__ __forceinline__ uint32_t woff(int n, int k) {
  return (uint32_t)(n & 7) * 16 + (uint32_t)(n >> 3) * SBO_W + (uint32_t)(k & 7) * 2 + (uint32_t)(k >> 3) * LBO_W;
}

// Epilogue of products A and B: W = D (+ cr when add), optionally sub -= W
// with cr holding sub's elements (C tiles in global memory), and W^T (three
// BF16 pieces) to the resident buffer for the next product.
__device__ void epilogue_w(uint32_t tmem, int n, int cw, const CRegs &cr, bool add, float *sub, unsigned char *smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = 32 * (warp & 3) + lane;
  const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int g = (warp >> 2) + 2 * e;
    if (g >= n / 16) continue;
    float v[16];
    tmem_sum16(tl + 16 * g, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = 16 * g + q;
      float x = 0.f;
      if (col < cw) {
        x = add ? v[q] + cr[e][q] : v[q];
        if (sub) __stcg(sub + (size_t)col * NB + m, cr[e][q] - x);
      }
      uint32_t p0, p1, p2;
      split3(x, p0, p1, p2);
      unsigned char *dst = smem + OFF_W + woff(col, m);
      *reinterpret_cast<unsigned short *>(dst) = (unsigned short)p0;
      *reinterpret_cast<unsigned short *>(dst + W_PC) = (unsigned short)p1;
      *reinterpret_cast<unsigned short *>(dst + 2 * W_PC) = (unsigned short)p2;
    }
  }
}

// Epilogue of a product that updates a C tile: c -= D (global memory), with
// cr holding c's elements.
__device__ void epilogue_c(uint32_t tmem, int n, int cw, float *c, const CRegs &cr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = 32 * (warp & 3) + lane;
  const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int g = (warp >> 2) + 2 * e;
    if (g >= n / 16) continue;
    float v[16];
    tmem_sum16(tl + 16 * g, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = 16 * g + q;
      if (col < cw) __stcg(c + (size_t)col * NB + m, cr[e][q] - v[q]);
    }
  }
}

// Order the epilogue's tensor-memory reads and shared-memory writes before
// the next product's MMAs (all threads).
__device__ __forceinline__ void between_products() {
  tc_fence_before();
  fence_async_smem();
  __syncthreads();
  tc_fence_after();
}

// One update task on a column slab of cw <= 128 columns (a whole tile, or a
// right-hand-side block).
//  mode: 1 UNMQR (V unit lower in tile V), 0 TSMQR (V = [I; V2], V2 the full
//        tile), 2 TTMQR (V2 the upper triangle of the tile)
//  trans: 1 applies Q^T, 0 applies Q
//  ct: top block (TS/TT; nullptr for UNMQR), cb: bottom block (or the
//      UNMQR target); both column-major with leading dimension 128, at the
//      slab's first column, in global memory
//  V: the reflector tile, Trec: the T record of the panel tile (the split
//     operand images written by the panel task, and the FP32 T when kept)
// Q^T (the direction of factorizations, least-squares plans and the server):
//   W = V^T C_b (+ C_t); C_t -= T^T W (TS / TT); C_b -= Y W with Y = V T^T
// from the panel's images. Q: W = V^T C_b (+ C_t); W' = T W; C_t -= W';
// C_b -= V W'.
// Returns false on a timeout.
__device__ bool update(int mode, int trans, const float *V, const float *Trec, float *ct, float *cb, int cw,
                       unsigned char *smem, State &st, Phases &ph, volatile int *abort, long long limit_ns) {
  const int n = (cw + 15) & ~15;
  const uint32_t tmem = st.tmem;
  const unsigned char *rec = reinterpret_cast<const unsigned char *>(Trec);
  const Src sva{V, NB, 0, NB, mode == 0 ? -1 : mode, 0};  // V^T (reflector, row): image REC_VA
  const Src scb{cb, NB, 0, cw, -1, 0};                     // C_b^T (column, row), from global memory
  const Src stt{Trec + REC_T32 / 4, NB, 1, NB, -1, 0};     // T (Q): gathered
  const Src svc{V, NB, 1, NB, mode == 0 ? -1 : mode, 0};  // V (row, reflector): image REC_VC (Q)
  fence_async_smem();  // earlier generic accesses of the stages before the bulk copies
  __syncthreads();
  if (threadIdx.x == 0) issue_image(rec + REC_VA, smem, OFF_RING_A, STAGE_A, st);
  Fetch f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) fetch_b(scb, c, f.b[c]);
  if (!product(sva, rec + REC_VA, &scb, trans ? nullptr : &stt, f, smem, st, ph, tmem, n, abort, limit_ns, true,
               false))
    return false;
  CRegs cr;
  load_c(ct, cw, cr);  // C_t (zeros for UNMQR) while product A's MMAs run
  if (!product_wait(st, ph, abort, limit_ns)) return false;
  if (trans) {
    // the next image (T^T, or Y for UNMQR) is requested while W^T is written; for TS / TT the
    // Y image follows into the same stages once the MMAs that read T^T completed
    fence_async_smem();
    __syncthreads();  // product A's stages are free (its MMAs completed) before the copies
    if (threadIdx.x == 0) issue_image(rec + (ct ? REC_TB : REC_Y), smem, OFF_RING_BC, STAGE_BC, st);
    epilogue_w(tmem, n, cw, cr, ct != nullptr, nullptr, smem);
    between_products();
    if (ct) {
      if (!product(sva, rec + REC_TB, nullptr, nullptr, f, smem, st, ph, tmem, n, abort, limit_ns, true))
        return false;
      fence_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) issue_image(rec + REC_Y, smem, OFF_RING_BC, STAGE_BC, st);
      epilogue_c(tmem, n, cw, ct, cr);  // C_t stayed in registers since epilogue A
      between_products();
    }
    if (!product(sva, rec + REC_Y, nullptr, nullptr, f, smem, st, ph, tmem, n, abort, limit_ns, true, false))
      return false;
    load_c(cb, cw, cr);  // C_b while the last product's MMAs run
    if (!product_wait(st, ph, abort, limit_ns)) return false;
    epilogue_c(tmem, n, cw, cb, cr);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return true;
  }
  epilogue_w(tmem, n, cw, cr, ct != nullptr, nullptr, smem);
  between_products();
  if (!product(stt, nullptr, nullptr, nullptr, f, smem, st, ph, tmem, n, abort, limit_ns)) return false;
  epilogue_w(tmem, n, cw, cr, false, ct, smem);  // cr still holds C_t
  between_products();
  if (!product(svc, rec + REC_VC, nullptr, nullptr, f, smem, st, ph, tmem, n, abort, limit_ns, false, false))
    return false;
  load_c(cb, cw, cr);
  if (!product_wait(st, ph, abort, limit_ns)) return false;
  epilogue_c(tmem, n, cw, cb, cr);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return true;
}

}  // namespace tc
}  // namespace hqr

namespace hqr {
namespace tc {

// ------------------------------------------------------------------ panel --
// GEQRT / TSQRT / TTQRT of one 128 x 128 FP32 tile (pair), unblocked, with
// the tile held in registers: warp w owns rows 16w .. 16w + 15, lane l owns
// columns l, l + 32, l + 64, l + 96. One Householder reflector per step
// (Householder convention of the scalar kernels: beta = -sign(alpha)
// ||(alpha, x)||, sign(+-0) = +1; a zero x gives the identity). A step needs
// one CTA barrier: each warp forms, over its own rows, the squared norm of
// column j and the products of column j with every other column; the
// partial sums meet in shared memory (double-buffered by step parity) and
// every thread finishes them in the same fixed order. The same products give
// the trailing-update coefficients (columns > j) and the Gram entries
// G(l, j) = v_l^T v_j (columns < j). T then follows from G: column by column
// within each 32 x 32 diagonal block (one warp per block, no CTA barrier),
// then by recursive doubling over the blocks: T([A B], [A B]) has T_AB =
// -T_A G_AB T_B (the compact-WY merge of two reflector blocks).
//
// Modes: 1 GE (the tile itself), 0 TS (R = upper triangle of the killer
// tile, X = the killed tile), 2 TT (X = upper triangle of the killed tile).
// Writes V / R back to the tiles, and the T record: the full T (zeros below
// the diagonal) and the split operand images of the updates.

constexpr int LDT = NB + 1;  // shared T / G array: T upper + diagonal, G(l, j) at (j, l)

struct PanelSmem {
  float tg[NB * LDT];        // also staging of the tile for loads
  float sv[NB * LDT];        // the factored tile (V and R), element (r, c) at c * LDT + r
  float rs[NB * (NB + 1) / 2];  // TS / TT: packed upper triangle of R, column c at c (c + 1) / 2
  float part[2][8][NB];      // per-warp partial products of column j with every column
  float pss[2][8];           // per-warp partial squared norms
  float pam[2][8];           // per-warp max |x| (scaled path)
  float prow[2][NB];         // GE: row j of the tile
  float tau[NB];
};
constexpr uint32_t PANEL_SMEM = sizeof(PanelSmem);

__device__ __forceinline__ int rsoff(int r, int c) { return c * (c + 1) / 2 + r; }

// Sums of the eight per-warp partials as a fixed tree (shorter dependence chain).
__device__ __forceinline__ float sum8s(const float *p, int stride) {
  const float a = p[0] + p[stride], b = p[2 * stride] + p[3 * stride];
  const float c = p[4 * stride] + p[5 * stride], d = p[6 * stride] + p[7 * stride];
  return (a + b) + (c + d);
}
__device__ __forceinline__ float sum8(const float *p) { return sum8s(p, 1); }

// Split image (chunk layout of the update stages) of a 128 x 128 operand
// whose element (m, k) is value(m, k); written once per panel tile. Piece
// (m, k group of 8): lanes take consecutive m.
template <typename F>
__device__ void write_image(unsigned char *dst, F value) {
#pragma unroll 1
  for (int u = 0; u < (NB * NB / 8) / NTHR; ++u) {
    const int p = threadIdx.x + NTHR * u;
    const int m = p & (NB - 1), kg = p >> 7;
    uint32_t w[NP][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t a0, a1, a2, b0, b1, b2;
      split3(value(m, 8 * kg + e), a0, a1, a2);
      split3(value(m, 8 * kg + e + 1), b0, b1, b2);
      w[0][e / 2] = a0 | (b0 << 16);
      w[1][e / 2] = a1 | (b1 << 16);
      w[2][e / 2] = a2 | (b2 << 16);
    }
    const uint32_t off = (uint32_t)(kg >> 2) * NP * A_PC + (uint32_t)(m & 7) * 16 + (uint32_t)(m >> 3) * SBO_C +
                         (uint32_t)(kg & 3) * LBO_C;
#pragma unroll
    for (int q = 0; q < NP; ++q)
      __stcg(reinterpret_cast<uint4 *>(dst + off + (uint32_t)q * A_PC), make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]));
  }
}

// Split image of Y = V T^T (element (m, k): row m of the tile, reflector k):
// Y(m, k) = sum over l >= k of V(m, l) T(k, l), V the masked reflectors of
// the factored tile `sv` (column l at l * LDT), T the upper triangle of `tg`
// (T(k, l) at k + l * LDT). Thread block: rows lane + 32 a (a < 4: the lanes
// of a warp read consecutive words) x 8 reflectors; warp w takes the
// reflector groups w and 15 - w (the same number of terms for every warp).
// FP32, with the terms in ascending l.
__device__ void write_y_image(int mode, const float *sv, const float *tg, unsigned char *dst) {
  constexpr int RB = 4;
#pragma unroll 1
  for (int u = 0; u < (NB / RB) * (NB / 8) / NTHR; ++u) {
    const int m0 = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int kg = u == 0 ? w : 15 - w;  // rows m0 + 32 a; warps: k groups w and 15 - w
    const int k0 = 8 * kg;
    float acc[RB][8];
#pragma unroll
    for (int a = 0; a < RB; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 2
    for (int l = k0; l < NB; ++l) {
      float v[RB], t[8];
#pragma unroll
      for (int a = 0; a < RB; ++a) v[a] = vmask(mode, m0 + 32 * a, l, sv[l * LDT + m0 + 32 * a]);
#pragma unroll
      for (int b = 0; b < 8; ++b) t[b] = k0 + b <= l ? tg[k0 + b + l * LDT] : 0.f;
#pragma unroll
      for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(v[a], t[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < RB; ++a) {
      const int m = m0 + 32 * a;
      uint32_t w[NP][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        uint32_t a0, a1, a2, b0, b1, b2;
        split3(acc[a][e], a0, a1, a2);
        split3(acc[a][e + 1], b0, b1, b2);
        w[0][e / 2] = a0 | (b0 << 16);
        w[1][e / 2] = a1 | (b1 << 16);
        w[2][e / 2] = a2 | (b2 << 16);
      }
      const uint32_t off = (uint32_t)(kg >> 2) * NP * A_PC + (uint32_t)(m & 7) * 16 + (uint32_t)(m >> 3) * SBO_C +
                           (uint32_t)(kg & 3) * LBO_C;
#pragma unroll
      for (int q = 0; q < NP; ++q)
        __stcg(reinterpret_cast<uint4 *>(dst + off + (uint32_t)q * A_PC),
               make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]));
    }
  }
}

// T of the 32 x 32 diagonal block d of the panel (warp d, d < 4), column by
// column: T(i, j) = -tau_j sum over i <= l < j of T(i, l) G(l, j), T(j, j) =
// tau_j, with G(l, j) = v_l^T v_j at (j, l) of `tg` and tau on its diagonal.
// Lane i keeps row i of the block in registers; the result replaces the
// block's upper triangle. These are the first five levels of the doubling
// (blocks of 1 .. 16 merged) without a CTA barrier.
__device__ __noinline__ void t_diag_block(float *tg) {
  const int d = threadIdx.x >> 5, i = threadIdx.x & 31, o = 32 * d;
  float tr[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float tau = tg[(o + j) * (LDT + 1)];
    float acc = 0.f;
#pragma unroll
    for (int l = 0; l < j; ++l)
      if (l >= i) acc = fmaf(tr[l], tg[(o + j) + (o + l) * LDT], acc);
    tr[j] = i < j ? -tau * acc : (i == j ? tau : 0.f);
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j)
    if (j >= i) tg[(o + i) + (o + j) * LDT] = tr[j];
}

// The remaining levels of the doubling (blocks of 32 and 64 merged): T_AB =
// -T_A (G_AB T_B), 4 x 4 output blocks per thread, T upper and G lower in
// `tg` as for t_diag_block. All threads; ends with a CTA barrier.
__device__ __noinline__ void t_merge_blocks(float *tg) {
  const int tid = threadIdx.x;
  for (int s = 32; s < NB; s *= 2) {
    const int nbk = s / 4, per = nbk * nbk, nblocks = (NB / (2 * s)) * per;
    const bool act = tid < nblocks;
    int a = 0, l0 = 0, j0 = 0;
    if (act) {
      const int pr = tid / per, rem = tid - pr * per;
      a = pr * 2 * s;
      l0 = a + (rem % nbk) * 4;
      j0 = a + s + (rem / nbk) * 4;
    }
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    if (act)  // X = G_AB T_B (T_B upper triangular: m <= j)
      for (int m = a + s; m <= j0 + 3; ++m) {
        float gv[4], tv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) gv[u] = tg[m + (l0 + u) * LDT];
#pragma unroll
        for (int v = 0; v < 4; ++v) tv[v] = m <= j0 + v ? tg[m + (j0 + v) * LDT] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(gv[u], tv[v], acc[u][v]);
      }
    __syncthreads();
    if (act)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) tg[(l0 + u) + (j0 + v) * LDT] = acc[u][v];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    if (act)  // T_AB = -T_A X (T_A upper triangular: m >= l)
      for (int m = l0; m < a + s; ++m) {
        float ta[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ta[u] = m >= l0 + u ? tg[(l0 + u) + m * LDT] : 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) xv[v] = tg[m + (j0 + v) * LDT];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(ta[u], xv[v], acc[u][v]);
      }
    __syncthreads();
    if (act)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) tg[(l0 + u) + (j0 + v) * LDT] = -acc[u][v];
    __syncthreads();
  }
}

__device__ void panel(int mode, float *X, float *Rg, float *Tg, bool with_t32, unsigned char *smem_raw) {
  PanelSmem &sm = *reinterpret_cast<PanelSmem *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rb = warp * 16;  // first row of this warp
  constexpr float tiny = 1e-30f, huge = 1e30f;
  // ---- load X (and R) through shared memory (coalesced)
  for (int e = tid; e < NB * NB; e += NTHR) {
    const int c = e >> 7, r = e & 127;
    float v = __ldcg(X + e);
    if (mode == 2 && r > c) v = 0.f;
    sm.tg[c * LDT + r] = v;
  }
  if (mode != 1)
    for (int e = tid; e < NB * NB; e += NTHR) {
      const int c = e >> 7, r = e & 127;
      if (r <= c) sm.rs[rsoff(r, c)] = __ldcg(Rg + e);
    }
  __syncthreads();
  float x[16][4];
#pragma unroll
  for (int i = 0; i < 16; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) x[i][q] = sm.tg[(lane + 32 * q) * LDT + rb + i];
  __syncthreads();
  // deferred R-row write of TS / TT (row j is read by every thread in step j)
  float prev_w[4] = {0.f, 0.f, 0.f, 0.f}, prev_r[4] = {0.f, 0.f, 0.f, 0.f}, prev_beta = 0.f;
  int prev_j = -1;
#pragma unroll
  for (int sj = 0; sj < 4; ++sj) {
    for (int jl = 0; jl < 32; ++jl) {
      const int j = 32 * sj + jl, buf = j & 1;
      // column j (this warp's rows), support masked
      float xv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float v = __shfl_sync(0xffffffffu, x[i][sj], jl);
        const int r = rb + i;
        const bool in = mode == 1 ? r > j : (mode == 2 ? r <= j : true);
        xv[i] = in ? v : 0.f;
      }
      float ss = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) ss = fmaf(xv[i], xv[i], ss);
      float d[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) s = fmaf(xv[i], x[i][q], s);
        d[q] = s;
        sm.part[buf][warp][lane + 32 * q] = s;
      }
      if (lane == 0) sm.pss[buf][warp] = ss;
      if (mode == 1 && warp == (j >> 4)) {  // row j of the tile (a jump on its register row)
        float *pr = sm.prow[buf] + lane;
        switch (j & 15) {
#define HQR_PROW(I) \
  case I:           \
    pr[0] = x[I][0]; \
    pr[32] = x[I][1]; \
    pr[64] = x[I][2]; \
    pr[96] = x[I][3]; \
    break;
          HQR_PROW(0) HQR_PROW(1) HQR_PROW(2) HQR_PROW(3) HQR_PROW(4) HQR_PROW(5) HQR_PROW(6) HQR_PROW(7)
          HQR_PROW(8) HQR_PROW(9) HQR_PROW(10) HQR_PROW(11) HQR_PROW(12) HQR_PROW(13) HQR_PROW(14) HQR_PROW(15)
#undef HQR_PROW
        }
      }
      __syncthreads();
      // R row of the previous step: every read of it happened before this barrier
      if (mode != 1 && warp == 0 && prev_j >= 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = lane + 32 * q;
          if (c > prev_j) sm.rs[rsoff(prev_j, c)] = prev_r[q] - prev_w[q];
        }
        if (lane == 0) sm.rs[rsoff(prev_j, prev_j)] = prev_beta;
      }
      const float sst = sum8(sm.pss[buf]);
      const float alpha = mode == 1 ? sm.prow[buf][j] : sm.rs[rsoff(j, j)];
      float snorm;
      bool rescaled = false;
      float am = 0.f;
      if (sst == 0.f) {
        snorm = 0.f;
      } else if (sst > tiny && sst < huge) {
        snorm = sqrtf(sst);
      } else {  // max-scaled second pass (uniform branch: every thread sees the same sums)
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) a = fmaxf(a, fabsf(xv[i]));
        if (lane == 0) sm.pam[buf][warp] = a;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 8; ++w) am = fmaxf(am, sm.pam[buf][w]);
        const float inv = 1.f / am;
        float s2 = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float t = xv[i] * inv;
          s2 = fmaf(t, t, s2);
        }
        // products again with the scaled column (no overflow in x^T a_c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < 16; ++i) s = fmaf(xv[i] * inv, x[i][q], s);
          d[q] = s;
        }
        __syncthreads();  // every thread has read the unscaled partials
#pragma unroll
        for (int q = 0; q < 4; ++q) sm.part[buf][warp][lane + 32 * q] = d[q];
        if (lane == 0) sm.pss[buf][warp] = s2;
        __syncthreads();
        float st2 = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) st2 += sm.pss[buf][w];
        snorm = am * sqrtf(st2);
        rescaled = true;
      }
      float beta = alpha, t = 0.f, scale = 0.f;
      if (snorm != 0.f) {
        // ||(alpha, x)||: the unscaled sum of squares plus alpha^2 when
        // neither can overflow, else hypot
        const float h = (!rescaled && fabsf(alpha) < 1e15f) ? sqrtf(fmaf(alpha, alpha, sst)) : hypotf(alpha, snorm);
        beta = alpha >= 0.f ? -h : h;
        t = (beta - alpha) / beta;
        scale = 1.f / (alpha - beta);
      }
      // the products' scale: x^T a_c = dsum (or am * dsum when rescaled)
      const float pscale = rescaled ? scale * am : scale;
      float wc[4], rowc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = lane + 32 * q;
        const float s = sum8s(&sm.part[buf][0][c], NB);
        rowc[q] = mode == 1 ? sm.prow[buf][c] : (c > j ? sm.rs[rsoff(j, c)] : 0.f);
        const float vta = rowc[q] + pscale * s;  // v_j^T a_c (GE, TS), v_j^T v_c for c < j
        wc[q] = c > j ? t * vta : 0.f;
        if (warp == 0 && c < j) sm.tg[j + c * LDT] = mode == 1 ? vta : pscale * s;  // G(c, j)
      }
      (void)d;
      if (tid == 0) sm.tau[j] = t;
      // apply the reflector to this thread's columns > j; column j becomes v
      float vf[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int r = rb + i;
        if (mode == 1)
          vf[i] = r > j ? xv[i] * scale : (r == j ? 1.f : 0.f);
        else
          vf[i] = xv[i] * scale;  // support already masked
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (lane + 32 * q > j)
#pragma unroll
          for (int i = 0; i < 16; ++i) x[i][q] = fmaf(-vf[i], wc[q], x[i][q]);
      if (lane == jl) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = rb + i;
          if (mode == 1) {
            if (r > j)
              x[i][sj] = vf[i];
            else if (r == j)
              x[i][sj] = beta;
          } else if (mode == 0 || r <= j) {
            x[i][sj] = vf[i];
          }
        }
      }
      if (mode != 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          prev_w[q] = wc[q];
          prev_r[q] = rowc[q];
        }
        prev_beta = beta;
        prev_j = j;
      }
    }
  }
  __syncthreads();
  if (mode != 1 && warp == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (c > prev_j) sm.rs[rsoff(prev_j, c)] = prev_r[q] - prev_w[q];
    }
    if (lane == 0) sm.rs[rsoff(prev_j, prev_j)] = prev_beta;
  }
  __syncthreads();
  // ---- T from G by recursive doubling
  for (int e = tid; e < NB; e += NTHR) sm.tg[e * LDT + e] = sm.tau[e];
  __syncthreads();
  if (warp < NB / 32) t_diag_block(sm.tg);
  __syncthreads();
  t_merge_blocks(sm.tg);
  // ---- the factored tile (V / R) to shared memory
#pragma unroll
  for (int i = 0; i < 16; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) sm.sv[(lane + 32 * q) * LDT + rb + i] = x[i][q];
  __syncthreads();
  // ---- write T (zeros below the diagonal, if kept) and the split images T^T, Y = V T^T
  unsigned char *rec = reinterpret_cast<unsigned char *>(Tg);
  if (with_t32)
    for (int e = tid; e < NB * NB; e += NTHR) {
      const int c = e >> 7, r = e & 127;
      __stcg(reinterpret_cast<float *>(rec + REC_T32) + e, r <= c ? sm.tg[r + c * LDT] : 0.f);
    }
  write_image(rec + REC_TB, [&](int m, int k) { return k <= m ? sm.tg[k + m * LDT] : 0.f; });
  write_y_image(mode, sm.sv, sm.tg, rec + REC_Y);
  // ---- V / R, and the split images V^T and V (masked to V's structure)
  for (int e = tid; e < NB * NB; e += NTHR) {
    const int c = e >> 7, r = e & 127;
    if (mode != 2 || r <= c) __stcg(X + e, sm.sv[c * LDT + r]);
    if (mode != 1 && r <= c) __stcg(Rg + e, sm.rs[rsoff(r, c)]);
  }
  write_image(rec + REC_VA, [&](int m, int k) { return vmask(mode, k, m, sm.sv[k + m * LDT]); });
  if (with_t32) write_image(rec + REC_VC, [&](int m, int k) { return vmask(mode, m, k, sm.sv[m + k * LDT]); });
  __syncthreads();
}

}  // namespace tc
}  // namespace hqr
