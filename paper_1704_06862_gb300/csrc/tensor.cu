// Tensor-core (tcgen05) contractions of the MLFMM for blocks of right-hand
// sides: leaf aggregation S_b = sum_{n in b} V_n (x) [eta0 c, v]_n as a dense
// product per leaf box, in split BF16 with FP32 accumulation in tensor memory.
//
// For one box with n bases, K directions and a pass of RB right-hand sides,
// the complex product S[(t,k)][(jm,r)] = sum_n V[n][t][k] X[n][jm][r] is the
// real product  D = A B  with
//   rows    m = 2 (t K + k) + ri        (4K rows: theta/phi, direction, re/im)
//   columns j = jm RB + r               (2 RB: J/M source, right-hand side)
//   inner   c = 2 n + ci                (2 n: basis, re/im of the coefficient)
//   A[m][c] = (ri, ci) = (0,0): Re V, (0,1): -Im V, (1,0): Im V, (1,1): Re V
//   B[c][j] = s_n Re x (ci = 0) or s_n Im x (ci = 1), x the coefficient of basis n.
// Each operand is split into three BF16 parts, a = a0 + a1 + a2 with
// a0 = bf16(a), a1 = bf16(a - a0), a2 = bf16(a - a0 - a1) (8 significant bits
// each, about 24 together), and D accumulates the six products a_i b_j with
// i + j <= 2 (the dropped terms are below 2^-26 of the product): FP32-level
// operands.  Two parts (three products, about 16 bits) are not enough here:
// the diagonal translations that follow add many plane-wave terms much larger
// than their sum (the more so the larger the truncation L), which amplified
// the 16-bit operands' error to 2e-4 of the whole product on a test cube.
//
// Mapping (one CTA per leaf box, 256 threads):
//   * A does not depend on the right-hand sides: it is split and laid out at
//     setup (k_agg_operand_build) in HBM in the exact shared-memory byte
//     layout, per box as chunks of (128-row tile, up to four k-steps, three
//     parts); the kernel streams the chunks with bulk asynchronous copies
//     (cp.async.bulk, completion counted in bytes on an mbarrier) into a
//     two-stage ring, the copy of chunk q + 1 in flight while the MMAs of
//     chunk q run;
//   * B (all k-steps of the box) is staged by the threads once per pass of
//     right-hand sides;
//   * one thread issues the MMAs (M = 128, N = 2 RB, K = 16, kind::f16 with
//     BF16 operands, both K-major, no swizzle) into a 128 x N FP32 tile in
//     tensor memory and commits them to an mbarrier; the waits on it are
//     bounded (SIE_ETIMEOUT's flag, then the CTA frees its tensor memory and
//     returns);
//   * the eight warps read the tile back (tcgen05.ld, warp w its lane
//     quarter w % 4 and column half w / 4) and write S.
// Shared-memory operand layout: the canonical no-swizzle K-major form, core
// matrices of 8 rows x 16 bytes (8 BF16 along K), 128 bytes each; within one
// k-step the two core matrices of a row group are 128 bytes apart (leading
// byte offset) and row groups 256 bytes apart (stride byte offset).
#include <cuda_bf16.h>

#include <map>
#include <mutex>

#include "common.h"

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of tcgen05.mma: start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit
// 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

// bulk asynchronous copy global -> shared, completion counted on an mbarrier:
// the issuing thread first announces the bytes (arrive + expect_tx)
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row, col) of a k-major operand tile stored as
// consecutive 16-wide k-steps of `rows` rows each (no-swizzle core matrices)
__device__ __forceinline__ uint32_t op_off(int row, int col, int rows) {
  const int s = col >> 4, cc = col & 15;
  return (uint32_t)(s * rows * 32 + (row >> 3) * 256 + (cc >> 3) * 128 + (row & 7) * 16 + (cc & 7) * 2);
}
// the three BF16 parts of v, stored at byte offset off of the parts' arrays
// (consecutive arrays `stride` bytes apart)
__device__ __forceinline__ void split_store(unsigned char *base, size_t stride, uint32_t off, float v) {
  const __nv_bfloat16 p0 = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(p0);
  const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
  const __nv_bfloat16 p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
  *reinterpret_cast<__nv_bfloat16 *>(base + off) = p0;
  *reinterpret_cast<__nv_bfloat16 *>(base + stride + off) = p1;
  *reinterpret_cast<__nv_bfloat16 *>(base + 2 * stride + off) = p2;
}

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;     // rows of one D tile
constexpr int TC_KCH = 4;     // k-steps per A chunk
constexpr int TC_PARTS = 3;   // BF16 parts per operand
constexpr int TC_KSTEP = TC_M * 32;                    // bytes of one part of one k-step of A (128 x 16 BF16)
constexpr int TC_STAGE = TC_PARTS * TC_KCH * TC_KSTEP;  // one ring stage: a whole chunk

// Layout of the pre-split A operand of one box (byte offsets from the box's
// start): chunk (row tile mt, chunk kc) at (mt ks + TC_KCH kc) TC_PARTS TC_KSTEP,
// holding its kn = min(TC_KCH, ks - TC_KCH kc) k-steps as [part][k-step][128 x 16]
// in the core-matrix layout of op_off.  ks = max(1, ceil(2 n / 16)).
__global__ void k_agg_operand_build(int K, const int *__restrict__ box_start, const int64_t *__restrict__ box_off,
                                    const cx<float> *__restrict__ V, unsigned char *__restrict__ A) {
  const int b = blockIdx.x, i0 = box_start[b], n = box_start[b + 1] - i0;
  const int ks = max(1, (2 * n + 15) >> 4), K2 = 2 * K, mtiles = (2 * K2 + TC_M - 1) / TC_M;
  unsigned char *base = A + box_off[b];
  const int per = 64 * 8;  // (row pair, basis) per (tile, k-step)
  for (int idx = threadIdx.x; idx < mtiles * ks * per; idx += blockDim.x) {
    const int ts = idx / per, e = idx - ts * per;
    const int mt = ts / ks, sg = ts - mt * ks;  // row tile, global k-step
    const int tkl = e >> 3, nbl = e & 7;
    const int tk = mt * 64 + tkl, nb = sg * 8 + nbl;
    float vr = 0.f, vi = 0.f;
    if (tk < K2 && nb < n) {
      const cx<float> v = V[(size_t)(i0 + nb) * K2 + tk];
      vr = v.re;
      vi = v.im;
    }
    const int kc = sg / TC_KCH, sl = sg - kc * TC_KCH, kn = min(TC_KCH, ks - kc * TC_KCH);
    unsigned char *chunk = base + (size_t)(mt * ks + kc * TC_KCH) * TC_PARTS * TC_KSTEP + (size_t)sl * TC_KSTEP;
    const size_t pstride = (size_t)kn * TC_KSTEP;  // between the parts of the chunk
    const int c = 2 * nbl;
    split_store(chunk, pstride, op_off(2 * tkl, c, TC_M), vr);
    split_store(chunk, pstride, op_off(2 * tkl, c + 1, TC_M), -vi);
    split_store(chunk, pstride, op_off(2 * tkl + 1, c, TC_M), vi);
    split_store(chunk, pstride, op_off(2 * tkl + 1, c + 1, TC_M), vr);
  }
}

// Leaf aggregation of one medium on the tensor cores, RB right-hand sides per
// pass (N = 2 RB columns).  ks_max: 16-wide k-steps of the largest box.
template <int RB>
__global__ void __launch_bounds__(TC_THREADS) k_aggregate_tc(int K, int ne, int nrhs, int ks_max,
                                                            const int *__restrict__ box_start,
                                                            const int64_t *__restrict__ box_off,
                                                            const int *__restrict__ basis_p,
                                                            const int *__restrict__ sign,
                                                            const unsigned char *__restrict__ Aop,
                                                            const cx<float> *__restrict__ x, cx<float> *__restrict__ S,
                                                            int wait_limit, int *err) {
  constexpr int N = 2 * RB;
  constexpr int NCOLS = N < 32 ? 32 : N;  // tensor-memory columns (a power of two >= 32)
  constexpr uint32_t IDESC = idesc_bf16_f32(TC_M, N);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const size_t bpart = (size_t)ks_max * N * 32;  // bytes of one part of B
  unsigned char *Bp = smem_raw;                    // [TC_PARTS][ks_max k-steps][N rows][16]
  unsigned char *ring = Bp + TC_PARTS * bpart;     // [2][TC_STAGE]
  __shared__ __align__(8) uint64_t full[2], mma_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x, i0 = box_start[b], n = box_start[b + 1] - i0;
  const int ks = max(1, (2 * n + 15) >> 4);  // k-steps of this box (an empty box: one step of zeros, D = 0)
  const int K2 = 2 * K;                      // (theta/phi, direction) pairs
  const int mtiles = (2 * K2 + TC_M - 1) / TC_M;
  const int nkc = (ks + TC_KCH - 1) / TC_KCH, nq = mtiles * nkc;  // chunks per pass
  const unsigned char *abox = Aop + box_off[b];
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&mma_done, 1);
    s_fail = 0;
  }
  if (warp == 0) tmem_alloc(&s_tmem, NCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  unsigned pf0 = 0, pf1 = 0, pm = 0;  // phases of the two ring stages and of the MMA barrier
  int issued = 0, consumed = 0;       // chunks copied in and used (thread 0's count is the one that matters)
  auto issue = [&](int q) {           // thread 0: chunk q into stage q & 1
    const int mt = q / nkc, kc = q - mt * nkc, kn = min(TC_KCH, ks - kc * TC_KCH);
    const uint32_t bytes = (uint32_t)(TC_PARTS * kn * TC_KSTEP);
    uint64_t *bar = &full[q & 1];
    mbar_expect_tx(bar, bytes);
    bulk_g2s(ring + (size_t)(q & 1) * TC_STAGE, abox + (size_t)(mt * ks + kc * TC_KCH) * TC_PARTS * TC_KSTEP, bytes,
             bar);
  };
  for (int r0 = 0; r0 < nrhs && !s_fail; r0 += RB) {
    const int nr = min(RB, nrhs - r0);
    // ---- B: all k-steps of the box, rows j = (jm, r), columns c = (basis, re/im)
    for (int idx = tid; idx < N * ks * 8; idx += TC_THREADS) {
      const int j = idx % N, cp = idx / N;  // cp: basis slot 0 .. 8 ks - 1
      const int jm = j / RB, r = j - jm * RB;
      float re = 0.f, im = 0.f;
      if (cp < n && r < nr) {
        const int p = basis_p[i0 + cp];
        const float sg = (float)sign[i0 + cp];
        const cx<float> v = x[((size_t)(r0 + r) * ne + p) * 2 + jm];
        re = sg * v.re;
        im = sg * v.im;
      }
      split_store(Bp, bpart, op_off(j, 2 * cp, N), re);
      split_store(Bp, bpart, op_off(j, 2 * cp + 1, N), im);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      issue(0);
      issued = 1;
      if (nq > 1) {
        issue(1);
        issued = 2;
      }
    }
    for (int q = 0; q < nq; ++q) {
      const int st = q & 1, mt = q / nkc, kc = q - mt * nkc, kn = min(TC_KCH, ks - kc * TC_KCH);
      const bool ok_full = mbar_wait(&full[st], st ? pf1 : pf0, wait_limit);
      if (ok_full) {  // a stage's phase advances only when its copy has arrived
        if (st) pf1 ^= 1u;
        else pf0 ^= 1u;
      }
      if (!ok_full) {
        if (lane == 0) atomicOr(err, 1);
        s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      consumed = q + 1;
      if (tid == 0) {
        tc_fence_after();
        const unsigned char *stage = ring + (size_t)st * TC_STAGE;
        for (int s = 0; s < kn; ++s) {
          // the six part products a_i b_j with i + j <= 2, smallest first
          for (int p6 = 0; p6 < 6; ++p6) {
            const int i = p6 < 3 ? 2 - p6 : (p6 < 5 ? 1 - (p6 - 3) : 0), jj = p6 < 3 ? p6 : (p6 < 5 ? p6 - 3 : 0);
            const uint64_t ad = smem_desc(smem_u32(stage + (size_t)(i * kn + s) * TC_KSTEP), 128, 256);
            const uint64_t bd = smem_desc(smem_u32(Bp + jj * bpart + (size_t)(kc * TC_KCH + s) * N * 32), 128, 256);
            tc_mma(tmem, ad, bd, IDESC, (kc > 0 || s > 0 || p6 > 0) ? 1 : 0);
          }
        }
        tc_commit(&mma_done);
      }
      const bool ok_mma = mbar_wait(&mma_done, pm, wait_limit);
      pm ^= 1u;
      if (!ok_mma) {
        if (lane == 0) atomicOr(err, 1);
        s_fail = 1;
      }
      tc_fence_after();
      // the stage is free: the next-but-one chunk goes into it
      if (tid == 0 && ok_mma && q + 2 < nq) {
        issue(q + 2);
        issued = q + 3;
      }
      __syncthreads();
      if (s_fail) break;
      if (kc < nkc - 1) continue;
      // ---- D tile -> S: warp w reads lanes 32 (w % 4) .. + 31, columns (w / 4) N/2 .. + N/2
      {
        const int m = 32 * (warp & 3) + lane, gm = mt * TC_M + m;
        const int tk = gm >> 1, ri = gm & 1;
        const int t = tk / K, k = tk - t * K;
        const int jc0 = (warp >> 2) * (N / 2);
        for (int c0 = 0; c0 < N / 2; c0 += 32) {
          float v[32];
          if (N / 2 >= 32) {
            tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(jc0 + c0), v);
          } else {
            // N / 2 = 16: read the 32 columns once (warps 0-3) and keep this half
            float w[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16), w);
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) v[qq] = w[jc0 + qq];
          }
          if (tk < K2) {
            const int cmax = min(32, N / 2 - c0);
            for (int qq = 0; qq < cmax; ++qq) {
              const int j = jc0 + c0 + qq, jm = j / RB, r = j - jm * RB;
              if (r < nr) {
                float *o = reinterpret_cast<float *>(S + ((size_t)b * 4 * nrhs + (size_t)(jm * 2 + t) * nrhs + r0 + r) * K + k);
                o[ri] = v[qq];
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // D read by every warp before the next tile's products overwrite it
      tc_fence_after();
    }
  }
  // after a wait gave up, copies and products may still be in flight: wait for
  // them (bounded again) before the shared and tensor memory are released
  if (s_fail && tid == 0) {
    // at most two chunks are outstanding, one per stage, each waited on its stage's pending phase
    for (int q = consumed; q < issued; ++q) mbar_wait(&full[q & 1], (q & 1) ? pf1 : pf0, wait_limit);
    mbar_wait(&mma_done, pm ^ 1u, wait_limit);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

template <int RB>
size_t agg_tc_smem(int max_leaf) {
  const int ks_max = std::max(1, (2 * max_leaf + 15) / 16);
  return (size_t)TC_PARTS * ks_max * (2 * RB) * 32 + 2 * (size_t)TC_STAGE;
}

template <int RB>
void launch_agg_tc(sie_ctx *c, int K, int nbox, int max_leaf, int nrhs, const int *box_start, const int64_t *box_off,
                   const int *basis_p, const int *sign, const unsigned char *Aop, const zf *x, zf *S, cudaStream_t st) {
  const int ks_max = std::max(1, (2 * max_leaf + 15) / 16);
  const size_t smem = agg_tc_smem<RB>(max_leaf);
  static bool raised[64] = {};
  int dev = 0;
  SIE_CUDA(cudaGetDevice(&dev));
  if (dev < 64 && !raised[dev]) {
    SIE_CUDA(cudaFuncSetAttribute(k_aggregate_tc<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    raised[dev] = true;
  }
  k_aggregate_tc<RB><<<nbox, TC_THREADS, smem, st>>>(K, c->ne, nrhs, ks_max, box_start, box_off, basis_p, sign, Aop,
                                                     x, S, c->wait_limit, c->d_err);
  SIE_CHECK_LAUNCH();
  c->launches++;
}

// ---------------------------------------------------------------- leaf receive
// For one box with n bases, a pass of RB right-hand sides and the box's
// incoming patterns I (J/M, theta/phi), the receive of the JMCFIE rows
//   y_J[p(n)] += cJ sum_(t,k) P[n][t][k] F1[t][k],  y_M[p(n)] -= cM sum_(t,k) P[n][t][k] F3[t][k]
// with the combined fields F1 = I^J - khat x I^M / eta, F3 = -eta khat x I^J - I^M
// (khat x (a_t, a_p) = (-a_p, a_t)) is the real product D = A B with
//   rows    m = 2 n + ri                  (the box's bases, re/im; 128-row tiles of 64 bases)
//   columns j = out RB + r                (out 0: J row, F1; out 1: M row, F3)
//   inner   c = 2 (t K + k) + ci          (4K: theta/phi, direction, re/im of F)
//   A[m][c] = the 2 x 2 real form of P[n][t][k] (as in the aggregation)
//   B[c][j] = Re F_out[t][k][r] (ci = 0) or Im F_out[t][k][r] (ci = 1).
// A (the receive patterns) is split at setup into the same chunked
// shared-memory layout as the aggregation operand and streamed by bulk
// copies; B is formed by the threads from I chunk by chunk (four k-steps =
// 32 (t, k) pairs), into a second buffer while the previous chunk's MMAs run.
__global__ void k_rec_operand_build(int K, const int *__restrict__ box_start, const int64_t *__restrict__ box_off,
                                    const cx<float> *__restrict__ P, unsigned char *__restrict__ A) {
  const int b = blockIdx.x, i0 = box_start[b], n = box_start[b + 1] - i0;
  const int K2 = 2 * K, ks = (2 * K2 + 15) >> 4, mtiles = max(1, (n + 63) >> 6);
  unsigned char *base = A + box_off[b];
  const int per = 64 * 8;  // (basis, direction pair) per (tile, k-step)
  for (int idx = threadIdx.x; idx < mtiles * ks * per; idx += blockDim.x) {
    const int ts = idx / per, e = idx - ts * per;
    const int mt = ts / ks, sg = ts - mt * ks;
    const int nl = e >> 3, tkl = e & 7;  // local basis (row pair), (t, k) pair within the k-step
    const int nb = mt * 64 + nl, tk = sg * 8 + tkl;
    float vr = 0.f, vi = 0.f;
    if (nb < n && tk < K2) {
      const cx<float> v = P[(size_t)(i0 + nb) * K2 + tk];
      vr = v.re;
      vi = v.im;
    }
    const int kc = sg / TC_KCH, sl = sg - kc * TC_KCH, kn = min(TC_KCH, ks - kc * TC_KCH);
    unsigned char *chunk = base + (size_t)(mt * ks + kc * TC_KCH) * TC_PARTS * TC_KSTEP + (size_t)sl * TC_KSTEP;
    const size_t pstride = (size_t)kn * TC_KSTEP;
    const int c = 2 * tkl;
    split_store(chunk, pstride, op_off(2 * nl, c, TC_M), vr);
    split_store(chunk, pstride, op_off(2 * nl, c + 1, TC_M), -vi);
    split_store(chunk, pstride, op_off(2 * nl + 1, c, TC_M), vi);
    split_store(chunk, pstride, op_off(2 * nl + 1, c + 1, TC_M), vr);
  }
}

// B of one chunk (k-steps kc TC_KCH .. + kn) of the receive: rows j = (out, r),
// columns c = 2 (t, k) + ci, three parts of (TC_KCH x N x 16) BF16 each
template <int RB>
__device__ __forceinline__ void rec_stage_b(unsigned char *Bc, int kc, int kn, int K, int nrhs, int r0, int nr,
                                            const cx<float> *__restrict__ Ib, cx<float> eta, cx<float> ieta) {
  constexpr int N = 2 * RB;
  const size_t bpart = (size_t)TC_KCH * N * 32;
  const int K2 = 2 * K;
  const size_t cs = (size_t)nrhs * K;
  for (int idx = threadIdx.x; idx < 8 * kn * RB; idx += TC_THREADS) {
    const int tkl = idx % (8 * kn), r = idx / (8 * kn);  // consecutive threads: consecutive directions
    const int tk = kc * TC_KCH * 8 + tkl;
    cx<float> f1, f3;
    if (tk < K2 && r < nr) {
      const int t = tk >= K ? 1 : 0, k = tk - t * K;
      const cx<float> *ib = Ib + (size_t)(r0 + r) * K + k;
      const cx<float> iJt = ib[0], iJp = ib[cs], iMt = ib[2 * cs], iMp = ib[3 * cs];
      f1 = t ? iJp - iMt * ieta : iJt + iMp * ieta;
      f3 = t ? -(eta * iJt) - iMp : eta * iJp - iMt;
    }
    const int c = 2 * tkl;
    split_store(Bc, bpart, op_off(r, c, N), f1.re);
    split_store(Bc, bpart, op_off(r, c + 1, N), f1.im);
    split_store(Bc, bpart, op_off(RB + r, c, N), f3.re);
    split_store(Bc, bpart, op_off(RB + r, c + 1, N), f3.im);
  }
}

// Leaf receive of one medium on the tensor cores, RB right-hand sides per pass;
// adds into y (FP32 product of the Krylov operator).  One CTA per leaf box.
template <int RB>
__global__ void __launch_bounds__(TC_THREADS) k_receive_tc(int K, int ne, int nrhs, const int *__restrict__ box_start,
                                                          const int64_t *__restrict__ box_off,
                                                          const int *__restrict__ basis_p,
                                                          const unsigned char *__restrict__ Aop,
                                                          const cx<float> *__restrict__ I, cx<float> eta,
                                                          cx<float> ieta, cx<float> cJ, cx<float> cM,
                                                          cx<float> *__restrict__ y, int wait_limit, int *err) {
  constexpr int N = 2 * RB;
  constexpr int NCOLS = N < 32 ? 32 : N;
  constexpr uint32_t IDESC = idesc_bf16_f32(TC_M, N);
  constexpr size_t BCH = (size_t)TC_PARTS * TC_KCH * N * 32;  // one B chunk buffer
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *ring = smem_raw;                 // [2][TC_STAGE]: A chunks
  unsigned char *Bbuf = ring + 2 * (size_t)TC_STAGE;  // [2][BCH]: B chunks
  __shared__ __align__(8) uint64_t full[2], mma_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x, i0 = box_start[b], n = box_start[b + 1] - i0;
  const int K2 = 2 * K, ks = (2 * K2 + 15) >> 4, nkc = (ks + TC_KCH - 1) / TC_KCH;
  const int mtiles = max(1, (n + 63) >> 6), nq = mtiles * nkc;
  const unsigned char *abox = Aop + box_off[b];
  const cx<float> *Ib = I + (size_t)b * 4 * nrhs * K;
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&mma_done, 1);
    s_fail = 0;
  }
  if (warp == 0) tmem_alloc(&s_tmem, NCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  unsigned pf0 = 0, pf1 = 0, pm = 0;
  int issued = 0, consumed = 0;
  auto issue = [&](int q) {  // thread 0: A chunk q into stage q & 1
    const int mt = q / nkc, kc = q - mt * nkc, kn = min(TC_KCH, ks - kc * TC_KCH);
    const uint32_t bytes = (uint32_t)(TC_PARTS * kn * TC_KSTEP);
    uint64_t *bar = &full[q & 1];
    mbar_expect_tx(bar, bytes);
    bulk_g2s(ring + (size_t)(q & 1) * TC_STAGE, abox + (size_t)(mt * ks + kc * TC_KCH) * TC_PARTS * TC_KSTEP, bytes,
             bar);
  };
  for (int r0 = 0; r0 < nrhs && !s_fail; r0 += RB) {
    const int nr = min(RB, nrhs - r0);
    if (tid == 0) {
      issue(0);
      issued = 1;
      if (nq > 1) {
        issue(1);
        issued = 2;
      }
    }
    rec_stage_b<RB>(Bbuf, 0, min(TC_KCH, ks), K, nrhs, r0, nr, Ib, eta, ieta);
    for (int q = 0; q < nq; ++q) {
      const int st = q & 1, mt = q / nkc, kc = q - mt * nkc, kn = min(TC_KCH, ks - kc * TC_KCH);
      fence_async_smem();  // this chunk's B (written by the threads) visible to the tensor cores
      const bool ok_full = mbar_wait(&full[st], st ? pf1 : pf0, wait_limit);
      if (ok_full) {
        if (st) pf1 ^= 1u;
        else pf0 ^= 1u;
      } else {
        if (lane == 0) atomicOr(err, 1);
        s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      consumed = q + 1;
      if (tid == 0) {
        tc_fence_after();
        const unsigned char *stage = ring + (size_t)st * TC_STAGE;
        const unsigned char *Bc = Bbuf + (size_t)st * BCH;
        for (int s = 0; s < kn; ++s)
          for (int p6 = 0; p6 < 6; ++p6) {
            const int i = p6 < 3 ? 2 - p6 : (p6 < 5 ? 1 - (p6 - 3) : 0), jj = p6 < 3 ? p6 : (p6 < 5 ? p6 - 3 : 0);
            const uint64_t ad = smem_desc(smem_u32(stage + (size_t)(i * kn + s) * TC_KSTEP), 128, 256);
            const uint64_t bd = smem_desc(smem_u32(Bc + (size_t)jj * TC_KCH * N * 32 + (size_t)s * N * 32), 128, 256);
            tc_mma(tmem, ad, bd, IDESC, (kc > 0 || s > 0 || p6 > 0) ? 1 : 0);
          }
        tc_commit(&mma_done);
      }
      // meanwhile the threads form the next chunk's B in the other buffer
      if (q + 1 < nq) {
        const int kc1 = (q + 1) % nkc;
        rec_stage_b<RB>(Bbuf + (size_t)((q + 1) & 1) * BCH, kc1, min(TC_KCH, ks - kc1 * TC_KCH), K, nrhs, r0, nr, Ib,
                        eta, ieta);
      }
      const bool ok_mma = mbar_wait(&mma_done, pm, wait_limit);
      pm ^= 1u;
      if (!ok_mma) {
        if (lane == 0) atomicOr(err, 1);
        s_fail = 1;
      }
      tc_fence_after();
      if (tid == 0 && ok_mma && q + 2 < nq) {
        issue(q + 2);
        issued = q + 3;
      }
      __syncthreads();
      if (s_fail) break;
      if (kc < nkc - 1) continue;
      // ---- D tile -> y: row m = 2 n + ri, the partner lane holds the other part
      {
        const int m = 32 * (warp & 3) + lane, nl = mt * 64 + (m >> 1), ri = m & 1;
        const int jc0 = (warp >> 2) * (N / 2);
        const int p = nl < n ? basis_p[i0 + nl] : 0;
        for (int c0 = 0; c0 < N / 2; c0 += 32) {
          float v[32];
          if (N / 2 >= 32) {
            tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(jc0 + c0), v);
          } else {
            float w[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16), w);
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) v[qq] = w[jc0 + qq];
          }
          const int cmax = min(32, N / 2 - c0);
          for (int qq = 0; qq < cmax; ++qq) {
            const float mine = v[qq], other = __shfl_xor_sync(0xffffffffu, mine, 1);
            const int j = jc0 + c0 + qq, out = j / RB, r = j - out * RB;
            if (ri == 0 && nl < n && r < nr) {
              const cx<float> sres(mine, other);
              cx<float> *o = y + ((size_t)(r0 + r) * ne + p) * 2 + out;
              if (out == 0) *o += cJ * sres;
              else *o -= cM * sres;
            }
          }
        }
      }
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }
  if (s_fail && tid == 0) {
    for (int q = consumed; q < issued; ++q) mbar_wait(&full[q & 1], (q & 1) ? pf1 : pf0, wait_limit);
    mbar_wait(&mma_done, pm ^ 1u, wait_limit);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

template <int RB>
constexpr size_t rec_tc_smem() {
  return 2 * (size_t)TC_STAGE + 2 * (size_t)TC_PARTS * TC_KCH * (2 * RB) * 32;
}

// ---------------------------------------------------------------- learned-preconditioner layers
// One dense layer of the learned preconditioner, C = act(X W^T + bias), with
// BF16 X [M][K] and W [N][K] (both K-major, the network's storage) and FP32
// accumulation in tensor memory: one CTA per (128-row tile of X, NT-column
// slice of W), the whole K (16 <= K <= 256, a multiple of 16) in one pass.
// The threads stage both operands into the no-swizzle core-matrix layout
// (16-byte pieces along K, eight loads in flight per thread); one thread
// issues the K/16 MMAs (M = 128, N = NT, K = 16) and commits them to an
// mbarrier (bounded wait, SIE_ETIMEOUT's flag); warp w reads lanes
// 32 (w % 4) .. + 31 and columns (w / 4) NT/2 .. + NT/2 back, adds the bias,
// applies max(0, .) if relu and writes FP32 (Cf) and/or BF16 (Cb) rows
// [M][N].  Rows past M are staged as zeros and not written.
template <int NT>
__global__ void __launch_bounds__(TC_THREADS) k_dense_tc(int M, int N, int K, const __nv_bfloat16 *__restrict__ X,
                                                        const __nv_bfloat16 *__restrict__ W,
                                                        const float *__restrict__ bias, int relu,
                                                        float *__restrict__ Cf, __nv_bfloat16 *__restrict__ Cb,
                                                        int wait_limit, int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *As = smem_raw;                     // [K/16 k-steps][128 rows][16 BF16]
  unsigned char *Bs = As + (size_t)K * TC_M * 2;    // [K/16 k-steps][NT rows][16 BF16]
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * NT;
  if (tid == 0) {
    mbar_init(&done, 1);
    s_fail = 0;
  }
  if (warp == 0) tmem_alloc(&s_tmem, NT);
  const int kp = K >> 3;  // 16-byte pieces per row
  constexpr int U = 8;    // loads in flight per thread
  // A: 128 rows of X, B: rows n0 .. n0 + NT - 1 of W; pieces 0 .. (128 + NT) kp - 1
  const int na = TC_M * kp, ntot = (TC_M + NT) * kp;
  for (int base = tid; base < ntot; base += TC_THREADS * U) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * TC_THREADS;
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (idx < na) {
        const int row = idx / kp, pc = idx - row * kp;
        if (m0 + row < M) v[u] = *reinterpret_cast<const uint4 *>(X + (size_t)(m0 + row) * K + 8 * pc);
      } else if (idx < ntot) {
        const int row = (idx - na) / kp, pc = (idx - na) - row * kp;
        v[u] = *reinterpret_cast<const uint4 *>(W + (size_t)(n0 + row) * K + 8 * pc);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * TC_THREADS;
      if (idx < na) {
        const int row = idx / kp, pc = idx - row * kp;
        *reinterpret_cast<uint4 *>(As + op_off(row, 8 * pc, TC_M)) = v[u];
      } else if (idx < ntot) {
        const int row = (idx - na) / kp, pc = (idx - na) - row * kp;
        *reinterpret_cast<uint4 *>(Bs + op_off(row, 8 * pc, NT)) = v[u];
      }
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr uint32_t IDESC = idesc_bf16_f32(TC_M, NT);
  if (tid == 0) {
    for (int s = 0; s < (K >> 4); ++s) {
      const uint64_t ad = smem_desc(smem_u32(As + (size_t)s * TC_M * 32), 128, 256);
      const uint64_t bd = smem_desc(smem_u32(Bs + (size_t)s * NT * 32), 128, 256);
      tc_mma(tmem, ad, bd, IDESC, s > 0 ? 1 : 0);
    }
    tc_commit(&done);
  }
  const bool ok = mbar_wait(&done, 0, wait_limit);
  if (!ok) {
    if (lane == 0) atomicOr(err, 1);
    s_fail = 1;
  }
  tc_fence_after();
  __syncthreads();
  if (!s_fail) {
    const int row = 32 * (warp & 3) + lane, gm = m0 + row, c0 = (warp >> 2) * (NT / 2);
    for (int cc = 0; cc < NT / 2; cc += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + cc), v);
      if (gm < M) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int col = n0 + c0 + cc + q;
          float y = v[q] + (bias ? bias[col] : 0.f);
          if (relu) y = fmaxf(y, 0.f);
          if (Cf) Cf[(size_t)gm * N + col] = y;
          if (Cb) Cb[(size_t)gm * N + col] = __float2bfloat16(y);
        }
      }
    }
  } else if (tid == 0) {
    mbar_wait(&done, 0, wait_limit);  // products possibly still in flight: bounded wait before release
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NT);
}

}  // namespace

// block size of the tensor-core aggregation for nrhs right-hand sides (0: not used)
int agg_tc_block(const sie_ctx *c, int nrhs) {
  if (c->agg_tc_min_rhs <= 0 || nrhs < c->agg_tc_min_rhs) return 0;
  if (c->agg_tc_rb) return c->agg_tc_rb;
  return nrhs >= 64 ? 64 : nrhs >= 32 ? 32 : 16;
}

// right-hand sides per pass of the tensor-core receive for a block of nrhs (0: the SIMT receive)
int rec_tc_block(const sie_ctx *c, int nrhs) {
  if (c->rec_tc_rb >= 0) return nrhs >= 2 ? c->rec_tc_rb : 0;
  if (nrhs < 16) return 0;
  return nrhs >= 64 ? 64 : nrhs >= 32 ? 32 : 16;
}

// pre-split A operand of the tensor-core aggregation for one medium (setup)
void build_agg_operand(sie_ctx *c, RegionHost &R, int K) {
  const int nbox = (int)R.box_start.size() - 1;
  if (nbox <= 0) return;
  const int K2 = 2 * K, mtiles = (2 * K2 + TC_M - 1) / TC_M;
  std::vector<int64_t> off(nbox + 1, 0);
  for (int b = 0; b < nbox; ++b) {
    const int n = R.box_start[b + 1] - R.box_start[b];
    const int ks = std::max(1, (2 * n + 15) / 16);
    off[b + 1] = off[b] + (int64_t)mtiles * ks * TC_PARTS * TC_KSTEP;
  }
  R.agg_op_bytes = (size_t)off[nbox];
  R.d_agg_off = dev_upload(c, off);
  R.d_agg_op = dev_alloc(c, R.agg_op_bytes);
  k_agg_operand_build<<<nbox, 256, 0, c->stream>>>(K, R.d_box_start, R.d_agg_off, (const zf *)R.d_V32,
                                                  (unsigned char *)R.d_agg_op);
  SIE_CHECK_LAUNCH();
  c->launches++;
}

bool op_aggregate_tc(sie_ctx *c, int rb, int K, int nbox, int max_leaf, int nrhs, const int *box_start,
                     const int64_t *box_off, const int *basis_p, const int *sign, const unsigned char *Aop,
                     const zf *x, zf *S, cudaStream_t st) {
  if (!Aop) return false;
  // fewer right-hand sides per pass while the largest box's operands do not fit in shared memory
  auto fits = [&](int r) {
    return (r == 64 ? agg_tc_smem<64>(max_leaf) : r == 32 ? agg_tc_smem<32>(max_leaf) : agg_tc_smem<16>(max_leaf)) <=
           200 * 1024;
  };
  while (rb > 16 && !fits(rb)) rb /= 2;
  if (!fits(rb)) return false;
  switch (rb) {
    case 16: launch_agg_tc<16>(c, K, nbox, max_leaf, nrhs, box_start, box_off, basis_p, sign, Aop, x, S, st); return true;
    case 32: launch_agg_tc<32>(c, K, nbox, max_leaf, nrhs, box_start, box_off, basis_p, sign, Aop, x, S, st); return true;
    case 64: launch_agg_tc<64>(c, K, nbox, max_leaf, nrhs, box_start, box_off, basis_p, sign, Aop, x, S, st); return true;
    default: return false;
  }
}

// pre-split A operand of the tensor-core receive for one medium (setup)
void build_rec_operand(sie_ctx *c, RegionHost &R, int K) {
  const int nbox = (int)R.box_start.size() - 1;
  if (nbox <= 0) return;
  const int ks = (4 * K + 15) / 16;
  std::vector<int64_t> off(nbox + 1, 0);
  for (int b = 0; b < nbox; ++b) {
    const int n = R.box_start[b + 1] - R.box_start[b];
    const int mtiles = std::max(1, (n + 63) / 64);
    off[b + 1] = off[b] + (int64_t)mtiles * ks * TC_PARTS * TC_KSTEP;
  }
  R.rec_op_bytes = (size_t)off[nbox];
  R.d_rec_off = dev_upload(c, off);
  R.d_rec_op = dev_alloc(c, R.rec_op_bytes);
  k_rec_operand_build<<<nbox, 256, 0, c->stream>>>(K, R.d_box_start, R.d_rec_off, (const zf *)R.d_P32,
                                                  (unsigned char *)R.d_rec_op);
  SIE_CHECK_LAUNCH();
  c->launches++;
}

bool op_receive_tc(sie_ctx *c, int rb, int K, int nbox, int nrhs, const int *box_start, const int64_t *box_off,
                   const int *basis_p, const unsigned char *Aop, const zf *I, zf eta, zf ieta, zf cJ, zf cM, zf *y,
                   cudaStream_t st) {
  if (!Aop) return false;
  auto go = [&](auto kern, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, bool> raised;
    int dev = 0;
    SIE_CUDA(cudaGetDevice(&dev));
    {
      std::lock_guard<std::mutex> lock(mu);
      bool &r = raised[{dev, reinterpret_cast<const void *>(kern)}];
      if (!r) {
        SIE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        r = true;
      }
    }
    kern<<<nbox, TC_THREADS, smem, st>>>(K, c->ne, nrhs, box_start, box_off, basis_p, Aop, I, eta, ieta, cJ, cM, y,
                                         c->wait_limit, c->d_err);
    SIE_CHECK_LAUNCH();
    c->launches++;
  };
  switch (rb) {
    case 16: go(k_receive_tc<16>, rec_tc_smem<16>()); return true;
    case 32: go(k_receive_tc<32>, rec_tc_smem<32>()); return true;
    case 64: go(k_receive_tc<64>, rec_tc_smem<64>()); return true;
    default: return false;
  }
}

// One learned-preconditioner layer on the tensor cores (k_dense_tc); false
// (nothing launched) for shapes or alignments it does not cover.
bool nn_dense_tc(sie_ctx *c, int M, int N, int K, const void *X, const void *W, const float *bias, int relu,
                 float *Cf, void *Cb) {
  constexpr int NT = 64;  // columns per CTA
  if (!c->nn_tc || M <= 0 || N <= 0 || N % NT || N / NT > 65535 || K < 16 || K > 256 || (K & 15)) return false;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(W) & 15)) return false;
  const size_t smem = (size_t)K * TC_M * 2 + (size_t)NT * K * 2;
  static std::mutex mu;
  static std::map<int, bool> raised;
  int dev = 0;
  SIE_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    bool &r = raised[dev];
    if (!r) {
      SIE_CUDA(cudaFuncSetAttribute(k_dense_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      r = true;
    }
  }
  k_dense_tc<NT><<<dim3((M + TC_M - 1) / TC_M, N / NT), TC_THREADS, smem, c->stream>>>(
      M, N, K, reinterpret_cast<const __nv_bfloat16 *>(X), reinterpret_cast<const __nv_bfloat16 *>(W), bias, relu, Cf,
      reinterpret_cast<__nv_bfloat16 *>(Cb), c->wait_limit, c->d_err);
  SIE_CHECK_LAUNCH();
  c->launches++;
  return true;
}
