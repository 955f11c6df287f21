// Hot path of the solver: y = Z x as near-field block-sparse product plus the
// MLFMM far field of every medium, and the ILU(0) preconditioner sweeps.
// Every kernel is templated on the real type: double (plain form) or float
// (mixed form, FP32 complex with FP32 accumulation).
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "common.h"

namespace {

template <typename T> struct tsel;
template <> struct tsel<double> {
  static void *near(sie_ctx *c) { return c->d_near64; }
  static void *V(RegionHost &R) { return R.d_V64; }
  static void *P(RegionHost &R) { return R.d_P64; }
  static void *Tr(LevelHost &L) { return L.d_T64; }
  static void *tp(LevelHost &L) { return L.d_tp64; }
  static void *Phi(LevelHost &L) { return L.d_Phi64; }
  static void *Thp(LevelHost &L) { return L.d_Thp64; }
  static void *Thm(LevelHost &L) { return L.d_Thm64; }
  static void *up(LevelHost &L) { return L.d_up64; }
  static void *dn(LevelHost &L) { return L.d_dn64; }
  static void *lo(IluHost &I) { return I.d_lo64; }
  static void *upv(IluHost &I) { return I.d_up64; }
  static void *tl(IluHost &I) { return I.d_tl64; }
  static void *tu(IluHost &I) { return I.d_tu64; }
};
template <> struct tsel<float> {
  static void *near(sie_ctx *c) { return c->d_near32; }
  static void *V(RegionHost &R) { return R.d_V32; }
  static void *P(RegionHost &R) { return R.d_P32; }
  static void *Tr(LevelHost &L) { return L.d_T32; }
  static void *tp(LevelHost &L) { return L.d_tp32; }
  static void *Phi(LevelHost &L) { return L.d_Phi32; }
  static void *Thp(LevelHost &L) { return L.d_Thp32; }
  static void *Thm(LevelHost &L) { return L.d_Thm32; }
  static void *up(LevelHost &L) { return L.d_up32; }
  static void *dn(LevelHost &L) { return L.d_dn32; }
  static void *lo(IluHost &I) { return I.d_lo32; }
  static void *upv(IluHost &I) { return I.d_up32; }
  static void *tl(IluHost &I) { return I.d_tl32; }
  static void *tu(IluHost &I) { return I.d_tu32; }
};

template <typename T>
__device__ __forceinline__ cx<T> shfl_down(cx<T> v, int d) {
  return cx<T>(__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d));
}
// the two unknowns (J, M) of one edge through the read-only path; p is 16-byte
// aligned (vectors start on 256-byte boundaries, an edge's pair is 2 complex)
// a value written by another CTA of the same launch: read through L2, not L1
__device__ __forceinline__ cx<float> ldcg_cx(const cx<float> *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return cx<float>(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldcg_cx(const cx<double> *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return cx<double>(v.x, v.y);
}
// the pair through L2 (ld.global.cg): for values written earlier in the same launch
__device__ __forceinline__ void ldcg_pair(const cx<float> *p, cx<float> &x0, cx<float> &x1) {
  const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
  x0 = cx<float>(v.x, v.y);
  x1 = cx<float>(v.z, v.w);
}
__device__ __forceinline__ void ldcg_pair(const cx<double> *p, cx<double> &x0, cx<double> &x1) {
  const double2 v0 = __ldcg(reinterpret_cast<const double2 *>(p)), v1 = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
  x0 = cx<double>(v0.x, v0.y);
  x1 = cx<double>(v1.x, v1.y);
}
__device__ __forceinline__ void ldg_pair(const cx<float> *p, cx<float> &x0, cx<float> &x1) {
  float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  x0 = cx<float>(v.x, v.y);
  x1 = cx<float>(v.z, v.w);
}
__device__ __forceinline__ void ldg_pair(const cx<double> *p, cx<double> &x0, cx<double> &x1) {
  double2 v0 = __ldg(reinterpret_cast<const double2 *>(p)), v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  x0 = cx<double>(v0.x, v0.y);
  x1 = cx<double>(v1.x, v1.y);
}
// z gathers of the ILU sweeps: a chained step reads values of earlier launches
// through the read-only path; the persistent kernel reads them through L2
template <bool CHAINED, typename T>
__device__ __forceinline__ void ldz_pair(const cx<T> *p, cx<T> &x0, cx<T> &x1) {
  if (CHAINED) ldg_pair(p, x0, x1);
  else ldcg_pair(p, x0, x1);
}
template <typename T>
__device__ __forceinline__ cx<T> warp_sum(cx<T> v) {
  for (int d = 16; d > 0; d >>= 1) v += shfl_down(v, d);
  return v;
}

// ---------------------------------------------------------------- near field
// y[p] (+)= sum_q B_pq x[q], 2x2 complex blocks (JJ, JM, MJ, MM); one warp per
// block row, lanes stride over the row's blocks (coalesced 16-byte loads).
template <typename T>
__global__ void k_near_spmv(int ne, int nrhs, const int *__restrict__ row_ptr, const int *__restrict__ col,
                            const cx<T> *__restrict__ B, const cx<T> *__restrict__ x, cx<T> *__restrict__ y,
                            int accumulate) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= ne) return;
  int s = row_ptr[warp], e = row_ptr[warp + 1];
  // a 2x2 complex block is 4 (FP32) or 8 (FP64) 8-byte words: read it as 16-byte vectors
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V16;
  constexpr int NV = (int)(4 * sizeof(cx<T>) / sizeof(V16));
  const V16 *Bv = reinterpret_cast<const V16 *>(B);
  for (int r = 0; r < nrhs; ++r) {
    const cx<T> *xr = x + (size_t)r * ne * 2;
    cx<T> a0, a1;
    int q = s + lane;
    // two blocks in flight per lane
    for (; q + 32 < e; q += 64) {
      int c0 = __ldg(col + q), c1 = __ldg(col + q + 32);
      V16 u0[NV], u1[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u0[v] = __ldg(Bv + (size_t)q * NV + v);
        u1[v] = __ldg(Bv + (size_t)(q + 32) * NV + v);
      }
      cx<T> xj0 = xr[2 * c0], xm0 = xr[2 * c0 + 1], xj1 = xr[2 * c1], xm1 = xr[2 * c1 + 1];
      const cx<T> *b0 = reinterpret_cast<const cx<T> *>(u0), *b1 = reinterpret_cast<const cx<T> *>(u1);
      a0 = cfma(b0[0], xj0, a0);
      a0 = cfma(b0[1], xm0, a0);
      a1 = cfma(b0[2], xj0, a1);
      a1 = cfma(b0[3], xm0, a1);
      a0 = cfma(b1[0], xj1, a0);
      a0 = cfma(b1[1], xm1, a0);
      a1 = cfma(b1[2], xj1, a1);
      a1 = cfma(b1[3], xm1, a1);
    }
    for (; q < e; q += 32) {
      int cc = __ldg(col + q);
      V16 u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = __ldg(Bv + (size_t)q * NV + v);
      const cx<T> *b = reinterpret_cast<const cx<T> *>(u);
      cx<T> xj = xr[2 * cc], xm = xr[2 * cc + 1];
      a0 = cfma(b[0], xj, a0);
      a0 = cfma(b[1], xm, a0);
      a1 = cfma(b[2], xj, a1);
      a1 = cfma(b[3], xm, a1);
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    if (lane == 0) {
      cx<T> *yr = y + ((size_t)r * ne + warp) * 2;
      if (accumulate) {
        yr[0] += a0;
        yr[1] += a1;
      } else {
        yr[0] = a0;
        yr[1] = a1;
      }
    }
  }
}

// Block of right-hand sides: each 2x2 block is loaded once and applied to RB
// right-hand sides at a time, so the matrix is read ceil(R/RB) times instead of R.
template <typename T, int RB>
__global__ void k_near_spmv_blk(int ne, int nrhs, const int *__restrict__ row_ptr, const int *__restrict__ col,
                                const cx<T> *__restrict__ B, const cx<T> *__restrict__ x, cx<T> *__restrict__ y,
                                int accumulate) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= ne) return;
  int s = row_ptr[warp], e = row_ptr[warp + 1];
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V16;
  constexpr int NV = (int)(4 * sizeof(cx<T>) / sizeof(V16));
  const V16 *Bv = reinterpret_cast<const V16 *>(B);
  const size_t vs = (size_t)ne * 2;
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int nr = min(RB, nrhs - r0);
    cx<T> a0[RB], a1[RB];
    for (int q = s + lane; q < e; q += 32) {
      int cc = __ldg(col + q);
      V16 u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = __ldg(Bv + (size_t)q * NV + v);
      const cx<T> *b = reinterpret_cast<const cx<T> *>(u);
#pragma unroll
      for (int rr = 0; rr < RB; ++rr)
        if (rr < nr) {
          const cx<T> *xr = x + (size_t)(r0 + rr) * vs;
          cx<T> xj = xr[2 * cc], xm = xr[2 * cc + 1];
          a0[rr] = cfma(b[0], xj, a0[rr]);
          a0[rr] = cfma(b[1], xm, a0[rr]);
          a1[rr] = cfma(b[2], xj, a1[rr]);
          a1[rr] = cfma(b[3], xm, a1[rr]);
        }
    }
#pragma unroll
    for (int rr = 0; rr < RB; ++rr)
      if (rr < nr) {
        cx<T> s0 = warp_sum(a0[rr]), s1 = warp_sum(a1[rr]);
        if (lane == 0) {
          cx<T> *yr = y + (size_t)(r0 + rr) * vs + 2 * (size_t)warp;
          if (accumulate) {
            yr[0] += s0;
            yr[1] += s1;
          } else {
            yr[0] = s0;
            yr[1] = s1;
          }
        }
      }
  }
}

// ---------------------------------------------------------------- async staging
// Per-thread 16-byte asynchronous global -> shared copies (cp.async), used to
// stream contiguous pattern blocks through a shared-memory ring: every thread
// issues its pieces of a chunk and commits them as one group; a chunk is read
// after cp.async.wait_group has retired its group and the CTA has synchronised.
__device__ __forceinline__ void cp_async16_s(void *smem, const void *gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_s() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_s() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// copy `bytes` (a multiple of 16, both addresses 16-byte aligned) with all threads of the CTA
__device__ __forceinline__ void cta_copy_async(void *dst, const void *src, size_t bytes) {
  char *d = reinterpret_cast<char *>(dst);
  const char *g = reinterpret_cast<const char *>(src);
  for (size_t o = (size_t)threadIdx.x * 16; o < bytes; o += (size_t)blockDim.x * 16) cp_async16_s(d + o, g + o);
}

// ---------------------------------------------------------------- MLFMM
// Leaf aggregation: S_b(k) = sum_{i in b} s_i [eta0 c, v]_p(i) (x) V_i(k).
// Every level's S and I are laid out [box][J/M][theta/phi][r][k]: for one
// right-hand side the K samples of a component are contiguous, so a warp over
// k reads and writes whole lines for any number of right-hand sides.
// One CTA per leaf box, threads over the directions k (up to KS per thread:
// 2, or 4 for the finely sampled leaves of strongly lossy media).  The box's patterns, one contiguous block, stream through shared
// memory in chunks of cb bases by asynchronous copies into a two-stage ring,
// so a whole chunk is in flight at once; the box's signed coefficients are
// staged in shared memory and each pattern value serves RB right-hand sides.
constexpr int STAGES = 2;
// single-RHS ILU sweep steps launched with programmatic dependent launch
constexpr bool ILU_PDL = true;
template <typename T, int RB, int KS>
__global__ void __launch_bounds__(256) k_aggregate(int K, int ne, int nrhs, int cb, const int *__restrict__ box_start,
                                                  const int *__restrict__ basis_p, const int *__restrict__ sign,
                                                  const cx<T> *__restrict__ V, const cx<T> *__restrict__ x,
                                                  cx<T> *__restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x, i0 = box_start[b], n = box_start[b + 1] - i0;
  const size_t per = (size_t)2 * K;  // complex values per basis
  cx<T> *ring = reinterpret_cast<cx<T> *>(smem_raw);       // [STAGES][cb][2][K]
  cx<T> *xs = ring + (size_t)STAGES * cb * per;            // [n][RB][2]
  const size_t cs = (size_t)nrhs * K;  // component stride
  const int nch = (n + cb - 1) / cb;
  auto fetch = [&](int ch) {  // every thread issues its pieces of chunk ch, then commits (possibly empty)
    if (ch < nch) {
      const int li0 = ch * cb, m = min(cb, n - li0);
      cta_copy_async(ring + (size_t)(ch % STAGES) * cb * per, V + (size_t)(i0 + li0) * per,
                     (size_t)m * per * sizeof(cx<T>));
    }
    cp_async_commit_s();
  };
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int nr = min(RB, nrhs - r0);
    for (int ch = 0; ch < STAGES; ++ch) fetch(ch);
    for (int idx = threadIdx.x; idx < n * RB; idx += blockDim.x) {
      const int li = idx / RB, rr = idx - li * RB;
      cx<T> xj, xm;
      if (rr < nr) {
        const int p = basis_p[i0 + li];
        const T sg = (T)sign[i0 + li];
        const cx<T> *xr = x + (size_t)(r0 + rr) * ne * 2;
        xj = sg * xr[2 * p];
        xm = sg * xr[2 * p + 1];
      }
      xs[2 * idx] = xj;
      xs[2 * idx + 1] = xm;
    }
    cx<T> a0[KS][RB], a1[KS][RB], a2[KS][RB], a3[KS][RB];
    for (int ch = 0; ch < nch; ++ch) {
      cp_async_wait_s<STAGES - 1>();
      __syncthreads();  // chunk ch (and, the first time, the coefficients) visible to all
      const int li0 = ch * cb, m = min(cb, n - li0);
      const cx<T> *v = ring + (size_t)(ch % STAGES) * cb * per;
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const int k = threadIdx.x + s * blockDim.x;
        if (k >= K) break;
        for (int li = 0; li < m; ++li) {
          const cx<T> vt = v[(size_t)li * per + k], vp = v[(size_t)li * per + K + k];
#pragma unroll
          for (int rr = 0; rr < RB; ++rr)
            if (rr < nr) {
              const cx<T> xj = xs[2 * ((li0 + li) * RB + rr)], xm = xs[2 * ((li0 + li) * RB + rr) + 1];
              a0[s][rr] = cfma(xj, vt, a0[s][rr]);
              a1[s][rr] = cfma(xj, vp, a1[s][rr]);
              a2[s][rr] = cfma(xm, vt, a2[s][rr]);
              a3[s][rr] = cfma(xm, vp, a3[s][rr]);
            }
        }
      }
      __syncthreads();  // the stage is free again
      fetch(ch + STAGES);
    }
    cp_async_wait_s<0>();
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      const int k = threadIdx.x + s * blockDim.x;
      if (k >= K) break;
#pragma unroll
      for (int rr = 0; rr < RB; ++rr)
        if (rr < nr) {
          cx<T> *o = S + ((size_t)b * 4 * nrhs + r0 + rr) * K + k;
          o[0] = a0[s][rr];
          o[cs] = a1[s][rr];
          o[2 * cs] = a2[s][rr];
          o[3 * cs] = a3[s][rr];
        }
    }
    __syncthreads();
  }
}

// Exact separable interpolation of one child's pattern to the parent
// sampling, shifted to the parent centre (upward pass).  One CTA per (child,
// right-hand side), JM of the sources J, M per pass.  The pattern is carried
// as three Cartesian components: (theta, phi) -> xyz at the child directions
// (A), trigonometric interpolation in phi (G = A Phi^T), the folded Lagrange
// step in theta (H = Th+ G + Th- G(phi + pi)), xyz -> (theta, phi) at the
// parent directions, times the shift exp(j k khat.(c_child - c_parent)).
// Output Y[child][J|M][theta|phi][r][k_parent]; k_up_sum adds the children.
// Register tiles: a G task owns the columns jp and jp + Np/2 of one theta row;
// an H task owns the pair (jp, jp + Np/2), whose phi + pi partners are each
// other, for two parent theta rows, so every shared-memory load feeds several FMAs.
template <typename T, int JM>
__global__ void __launch_bounds__(256) k_interp_up(int Kc, int Lc, int Kp, int Lp, int nrhs,
                                                  const int *__restrict__ oct, const T *__restrict__ tpc,
                                                  const T *__restrict__ tpp, const T *__restrict__ Phi,
                                                  const T *__restrict__ Thp, const T *__restrict__ Thm,
                                                  const cx<T> *__restrict__ up, const cx<T> *__restrict__ Sc,
                                                  cx<T> *__restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int Q = 3 * JM, IP = 2;
  const int Nc = 2 * Lc + 2, Np = 2 * Lp + 2, nthc = Lc + 1, nthp = Lp + 1, hp = Lp + 1;
  cx<T> *A = reinterpret_cast<cx<T> *>(smem_raw);  // [Q][Kc]
  cx<T> *G = A + (size_t)Q * Kc;                    // [Q][nthc][Np]
  T *PhT = reinterpret_cast<T *>(G + (size_t)Q * nthc * Np);  // [Nc][Np]
  T *Tps = PhT + Nc * Np, *Tms = Tps + nthp * nthc;           // [nthp][nthc]
  const int c = blockIdx.x, r = blockIdx.y, o = oct[c], tid = threadIdx.x, NT = blockDim.x;
  for (int i = tid; i < Np * Nc; i += NT) {
    const int jp = i / Nc, jc = i - jp * Nc;
    PhT[jc * Np + jp] = Phi[i];
  }
  for (int i = tid; i < nthp * nthc; i += NT) {
    Tps[i] = Thp[i];
    Tms[i] = Thm[i];
  }
  const int nib = (nthp + IP - 1) / IP;
  // with gridDim.z = 2 each CTA takes one of the sources (J, M), else both in turn
  const int jm_beg = gridDim.z > 1 ? (int)blockIdx.z * JM : 0, jm_end = gridDim.z > 1 ? jm_beg + JM : 2;
  for (int jm0 = jm_beg; jm0 < jm_end; jm0 += JM) {
    __syncthreads();
    for (int i = tid; i < JM * Kc; i += NT) {
      const int m = i / Kc, t = i - m * Kc;
      const cx<T> *st = Sc + (((size_t)c * 4 + (jm0 + m) * 2) * nrhs + r) * Kc;
      const cx<T> ft = st[t], fp = st[(size_t)nrhs * Kc + t];
      const T *u = tpc + 6 * (size_t)t;
#pragma unroll
      for (int x = 0; x < 3; ++x) A[(size_t)(m * 3 + x) * Kc + t] = ft * u[x] + fp * u[3 + x];
    }
    __syncthreads();
    for (int task = tid; task < nthc * hp; task += NT) {
      const int ic = task / hp, jp = task - ic * hp;
      cx<T> g0[Q], g1[Q];
      for (int jc = 0; jc < Nc; ++jc) {
        const T f0 = PhT[jc * Np + jp], f1 = PhT[jc * Np + jp + hp];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const cx<T> a = A[(size_t)q * Kc + ic * Nc + jc];
          g0[q].re = fma(f0, a.re, g0[q].re);
          g0[q].im = fma(f0, a.im, g0[q].im);
          g1[q].re = fma(f1, a.re, g1[q].re);
          g1[q].im = fma(f1, a.im, g1[q].im);
        }
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        G[((size_t)q * nthc + ic) * Np + jp] = g0[q];
        G[((size_t)q * nthc + ic) * Np + jp + hp] = g1[q];
      }
    }
    __syncthreads();
    for (int task = tid; task < nib * hp; task += NT) {
      const int ib = task / hp, jh = task - ib * hp, ip0 = ib * IP;
      cx<T> h0[IP][Q], h1[IP][Q];  // parent columns jh and jh + hp
      for (int ic = 0; ic < nthc; ++ic) {
        cx<T> ga[Q], gb[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          ga[q] = G[((size_t)q * nthc + ic) * Np + jh];
          gb[q] = G[((size_t)q * nthc + ic) * Np + jh + hp];
        }
#pragma unroll
        for (int k = 0; k < IP; ++k) {
          const int ip = min(ip0 + k, nthp - 1);
          const T a = Tps[ip * nthc + ic], bq = Tms[ip * nthc + ic];
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            h0[k][q].re = fma(a, ga[q].re, fma(bq, gb[q].re, h0[k][q].re));
            h0[k][q].im = fma(a, ga[q].im, fma(bq, gb[q].im, h0[k][q].im));
            h1[k][q].re = fma(a, gb[q].re, fma(bq, ga[q].re, h1[k][q].re));
            h1[k][q].im = fma(a, gb[q].im, fma(bq, ga[q].im, h1[k][q].im));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < IP; ++k) {
        const int ip = ip0 + k;
        if (ip >= nthp) break;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int tp = ip * Np + jh + half * hp;
          const T *u = tpp + 6 * (size_t)tp;
          const cx<T> sh = up[(size_t)o * Kp + tp];
#pragma unroll
          for (int m = 0; m < JM; ++m) {
            const cx<T> *H = half ? &h1[k][3 * m] : &h0[k][3 * m];
            const cx<T> yt = H[0] * u[0] + H[1] * u[1] + H[2] * u[2];
            const cx<T> yp = H[0] * u[3] + H[1] * u[4] + H[2] * u[5];
            Y[(((size_t)c * 4 + (jm0 + m) * 2) * nrhs + r) * Kp + tp] = sh * yt;
            Y[(((size_t)c * 4 + (jm0 + m) * 2 + 1) * nrhs + r) * Kp + tp] = sh * yp;
          }
        }
      }
    }
  }
}

// Chunked form of k_interp_up for parent samplings too large for shared memory.
// The parent's column pairs (jp, jp + Np/2) are taken cw at a time (a chunk:
// G holds only its 2 cw columns), so a large parent sampling fits in shared
// memory; with one chunk (cw = Np/2) the arithmetic is that of a single pass.
// GT: the interpolation tables are read from global memory (through L1)
// instead of shared memory, for the electrically large boxes of dense media
// whose child pattern and tables together exceed it; same arithmetic.
template <typename T, int JM, bool GT>
__global__ void __launch_bounds__(256) k_interp_up_chunked(int Kc, int Lc, int Kp, int Lp, int nrhs, int cw_max,
                                                  const int *__restrict__ oct, const T *__restrict__ tpc,
                                                  const T *__restrict__ tpp, const T *__restrict__ Phi,
                                                  const T *__restrict__ Thp, const T *__restrict__ Thm,
                                                  const cx<T> *__restrict__ up, const cx<T> *__restrict__ Sc,
                                                  cx<T> *__restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int Q = 3 * JM, IP = 2;
  const int Nc = 2 * Lc + 2, Np = 2 * Lp + 2, nthc = Lc + 1, nthp = Lp + 1, hp = Lp + 1;
  const int CW = cw_max, G2 = 2 * cw_max;           // chunk width (column pairs), G row length
  cx<T> *A = reinterpret_cast<cx<T> *>(smem_raw);  // [Q][Kc]
  cx<T> *G = A + (size_t)Q * Kc;                    // [Q][nthc][2 CW]: pair (jp, jp + hp) at (jl, CW + jl)
  T *PhT = reinterpret_cast<T *>(G + (size_t)Q * nthc * G2);  // [Nc][Np]
  T *Tps = PhT + Nc * Np, *Tms = Tps + nthp * nthc;            // [nthp][nthc]
  const int c = blockIdx.x, r = blockIdx.y, o = oct[c], tid = threadIdx.x, NT = blockDim.x;
  if (!GT) {
    for (int i = tid; i < Np * Nc; i += NT) {
      const int jp = i / Nc, jc = i - jp * Nc;
      PhT[jc * Np + jp] = Phi[i];
    }
    for (int i = tid; i < nthp * nthc; i += NT) {
      Tps[i] = Thp[i];
      Tms[i] = Thm[i];
    }
  }
  const T *Tpa = GT ? Thp : Tps, *Tma = GT ? Thm : Tms;
  const int nib = (nthp + IP - 1) / IP;
  // with gridDim.z = 2 each CTA takes one of the sources (J, M), else both in turn
  const int jm_beg = gridDim.z > 1 ? (int)blockIdx.z * JM : 0, jm_end = gridDim.z > 1 ? jm_beg + JM : 2;
  for (int jm0 = jm_beg; jm0 < jm_end; jm0 += JM) {
    __syncthreads();
    for (int i = tid; i < JM * Kc; i += NT) {
      const int m = i / Kc, t = i - m * Kc;
      const cx<T> *st = Sc + (((size_t)c * 4 + (jm0 + m) * 2) * nrhs + r) * Kc;
      const cx<T> ft = st[t], fp = st[(size_t)nrhs * Kc + t];
      const T *u = tpc + 6 * (size_t)t;
#pragma unroll
      for (int x = 0; x < 3; ++x) A[(size_t)(m * 3 + x) * Kc + t] = ft * u[x] + fp * u[3 + x];
    }
    for (int j0 = 0; j0 < hp; j0 += CW) {
      const int cw = min(CW, hp - j0);
      __syncthreads();  // A complete; G free again
      for (int task = tid; task < nthc * cw; task += NT) {
        const int ic = task / cw, jl = task - ic * cw, jp = j0 + jl;
        cx<T> g0[Q], g1[Q];
        for (int jc = 0; jc < Nc; ++jc) {
          const T f0 = GT ? Phi[(size_t)jp * Nc + jc] : PhT[jc * Np + jp];
          const T f1 = GT ? Phi[(size_t)(jp + hp) * Nc + jc] : PhT[jc * Np + jp + hp];
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const cx<T> a = A[(size_t)q * Kc + ic * Nc + jc];
            g0[q].re = fma(f0, a.re, g0[q].re);
            g0[q].im = fma(f0, a.im, g0[q].im);
            g1[q].re = fma(f1, a.re, g1[q].re);
            g1[q].im = fma(f1, a.im, g1[q].im);
          }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          G[((size_t)q * nthc + ic) * G2 + jl] = g0[q];
          G[((size_t)q * nthc + ic) * G2 + CW + jl] = g1[q];
        }
      }
      __syncthreads();
      for (int task = tid; task < nib * cw; task += NT) {
        const int ib = task / cw, jl = task - ib * cw, jh = j0 + jl, ip0 = ib * IP;
        cx<T> h0[IP][Q], h1[IP][Q];  // parent columns jh and jh + hp
        for (int ic = 0; ic < nthc; ++ic) {
          cx<T> ga[Q], gb[Q];
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            ga[q] = G[((size_t)q * nthc + ic) * G2 + jl];
            gb[q] = G[((size_t)q * nthc + ic) * G2 + CW + jl];
          }
#pragma unroll
          for (int k = 0; k < IP; ++k) {
            const int ip = min(ip0 + k, nthp - 1);
            const T a = Tpa[ip * nthc + ic], bq = Tma[ip * nthc + ic];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
              h0[k][q].re = fma(a, ga[q].re, fma(bq, gb[q].re, h0[k][q].re));
              h0[k][q].im = fma(a, ga[q].im, fma(bq, gb[q].im, h0[k][q].im));
              h1[k][q].re = fma(a, gb[q].re, fma(bq, ga[q].re, h1[k][q].re));
              h1[k][q].im = fma(a, gb[q].im, fma(bq, ga[q].im, h1[k][q].im));
            }
          }
        }
#pragma unroll
        for (int k = 0; k < IP; ++k) {
          const int ip = ip0 + k;
          if (ip >= nthp) break;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int tp = ip * Np + jh + half * hp;
            const T *u = tpp + 6 * (size_t)tp;
            const cx<T> sh = up[(size_t)o * Kp + tp];
#pragma unroll
            for (int m = 0; m < JM; ++m) {
              const cx<T> *H = half ? &h1[k][3 * m] : &h0[k][3 * m];
              const cx<T> yt = H[0] * u[0] + H[1] * u[1] + H[2] * u[2];
              const cx<T> yp = H[0] * u[3] + H[1] * u[4] + H[2] * u[5];
              Y[(((size_t)c * 4 + (jm0 + m) * 2) * nrhs + r) * Kp + tp] = sh * yt;
              Y[(((size_t)c * 4 + (jm0 + m) * 2 + 1) * nrhs + r) * Kp + tp] = sh * yp;
            }
          }
        }
      }
    }
  }
}

// S_parent = sum over children of the shifted, interpolated child patterns.
template <typename T>
__global__ void k_up_sum(int Kp, int nrhs, const int *__restrict__ ch_ptr, const int *__restrict__ ch_idx,
                         const cx<T> *__restrict__ Y, cx<T> *__restrict__ Sp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (t >= Kp) return;
  const int s0 = ch_ptr[b], s1 = ch_ptr[b + 1];
  const size_t cs = (size_t)nrhs * Kp;  // component stride
  for (int r = 0; r < nrhs; ++r) {
    // the four components of a child loaded together, children in order
    cx<T> a0, a1, a2, a3;
#pragma unroll 4
    for (int s = s0; s < s1; ++s) {
      const cx<T> *y = Y + ((size_t)ch_idx[s] * 4 * nrhs + r) * Kp + t;
      a0 += y[0];
      a1 += y[cs];
      a2 += y[2 * cs];
      a3 += y[3 * cs];
    }
    cx<T> *o = Sp + ((size_t)b * 4 * nrhs + r) * Kp + t;
    o[0] = a0;
    o[cs] = a1;
    o[2 * cs] = a2;
    o[3 * cs] = a3;
  }
}

// Exact transpose of k_interp_up (anterpolation, downward pass), with the
// receive shift exp(-j k khat.(c_child - c_parent)): one CTA per (child box,
// right-hand side), I_child += Interp^T [dn (.) I_parent].  Quadrature weights
// are folded into the translators, so the adjoint is the plain transpose.
// Register tiles as in k_interp_up: a theta-step task owns the column pair
// (j, j + Np/2) for two child theta rows; a phi-step task owns the child
// columns jc and jc + Nc/2 of one theta row.
template <typename T, int JM>
__global__ void __launch_bounds__(256) k_anterp_dn(int Kc, int Lc, int Kp, int Lp, int nrhs,
                                                  const int *__restrict__ parent, const int *__restrict__ oct,
                                                  const T *__restrict__ tpc, const T *__restrict__ tpp,
                                                  const T *__restrict__ Phi, const T *__restrict__ Thp,
                                                  const T *__restrict__ Thm, const cx<T> *__restrict__ dn,
                                                  const cx<T> *__restrict__ Ip, cx<T> *__restrict__ Ic) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int Q = 3 * JM, IC = 2;
  const int Nc = 2 * Lc + 2, Np = 2 * Lp + 2, nthc = Lc + 1, nthp = Lp + 1, hp = Lp + 1, hc = Lc + 1;
  cx<T> *A = reinterpret_cast<cx<T> *>(smem_raw);  // [Q][Kp]
  cx<T> *G = A + (size_t)Q * Kp;                    // [Q][nthc][Np]
  T *Ps = reinterpret_cast<T *>(G + (size_t)Q * nthc * Np);  // Phi [Np][Nc]
  T *Tps = Ps + Np * Nc, *Tms = Tps + nthp * nthc;           // [nthp][nthc]
  const int c = blockIdx.x, r = blockIdx.y, pb = parent[c], o = oct[c], tid = threadIdx.x, NT = blockDim.x;
  for (int i = tid; i < Np * Nc; i += NT) Ps[i] = Phi[i];
  for (int i = tid; i < nthp * nthc; i += NT) {
    Tps[i] = Thp[i];
    Tms[i] = Thm[i];
  }
  const int nicb = (nthc + IC - 1) / IC;
  // with gridDim.z = 2 each CTA takes one of the sources (J, M), else both in turn
  const int jm_beg = gridDim.z > 1 ? (int)blockIdx.z * JM : 0, jm_end = gridDim.z > 1 ? jm_beg + JM : 2;
  for (int jm0 = jm_beg; jm0 < jm_end; jm0 += JM) {
    __syncthreads();
    for (int i = tid; i < JM * Kp; i += NT) {
      const int m = i / Kp, t = i - m * Kp;
      const cx<T> *it = Ip + (((size_t)pb * 4 + (jm0 + m) * 2) * nrhs + r) * Kp;
      const cx<T> sh = dn[(size_t)o * Kp + t];
      const cx<T> ut = sh * it[t], up_ = sh * it[(size_t)nrhs * Kp + t];
      const T *u = tpp + 6 * (size_t)t;
#pragma unroll
      for (int x = 0; x < 3; ++x) A[(size_t)(m * 3 + x) * Kp + t] = ut * u[x] + up_ * u[3 + x];
    }
    __syncthreads();
    // transpose of the theta step: G[q][ic][j] = sum_ip Th+[ip][ic] A[q][ip][j] + Th-[ip][ic] A[q][ip][j + Np/2]
    for (int task = tid; task < nicb * hp; task += NT) {
      const int cb = task / hp, jh = task - cb * hp, ic0 = cb * IC;
      cx<T> g0[IC][Q], g1[IC][Q];
      for (int ip = 0; ip < nthp; ++ip) {
        cx<T> aa[Q], ab[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          aa[q] = A[(size_t)q * Kp + ip * Np + jh];
          ab[q] = A[(size_t)q * Kp + ip * Np + jh + hp];
        }
#pragma unroll
        for (int k = 0; k < IC; ++k) {
          const int ic = min(ic0 + k, nthc - 1);
          const T w1 = Tps[ip * nthc + ic], w2 = Tms[ip * nthc + ic];
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            g0[k][q].re = fma(w1, aa[q].re, fma(w2, ab[q].re, g0[k][q].re));
            g0[k][q].im = fma(w1, aa[q].im, fma(w2, ab[q].im, g0[k][q].im));
            g1[k][q].re = fma(w1, ab[q].re, fma(w2, aa[q].re, g1[k][q].re));
            g1[k][q].im = fma(w1, ab[q].im, fma(w2, aa[q].im, g1[k][q].im));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < IC; ++k) {
        const int ic = ic0 + k;
        if (ic >= nthc) break;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          G[((size_t)q * nthc + ic) * Np + jh] = g0[k][q];
          G[((size_t)q * nthc + ic) * Np + jh + hp] = g1[k][q];
        }
      }
    }
    __syncthreads();
    // transpose of the phi step, projection to (theta, phi) at the child directions
    for (int task = tid; task < nthc * hc; task += NT) {
      const int ic = task / hc, jc = task - ic * hc;
      cx<T> c0[Q], c1[Q];
      for (int jp = 0; jp < Np; ++jp) {
        const T f0 = Ps[jp * Nc + jc], f1 = Ps[jp * Nc + jc + hc];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const cx<T> g = G[((size_t)q * nthc + ic) * Np + jp];
          c0[q].re = fma(f0, g.re, c0[q].re);
          c0[q].im = fma(f0, g.im, c0[q].im);
          c1[q].re = fma(f1, g.re, c1[q].re);
          c1[q].im = fma(f1, g.im, c1[q].im);
        }
      }
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int tc = ic * Nc + jc + half * hc;
        const T *u = tpc + 6 * (size_t)tc;
#pragma unroll
        for (int m = 0; m < JM; ++m) {
          const cx<T> *C = half ? &c1[3 * m] : &c0[3 * m];
          cx<T> *it = Ic + (((size_t)c * 4 + (jm0 + m) * 2) * nrhs + r) * Kc;
          it[tc] += C[0] * u[0] + C[1] * u[1] + C[2] * u[2];
          it[(size_t)nrhs * Kc + tc] += C[0] * u[3] + C[1] * u[4] + C[2] * u[5];
        }
      }
    }
  }
}

// Chunked form of k_anterp_dn for parent samplings too large for shared memory.
// The parent's column pairs are taken cw at a time (a chunk of A and G in
// shared memory); each chunk adds its part of the phi-transpose sums into the
// child, columns jp of the chunk first, then their partners jp + Np/2 (with
// one chunk, the order of a single pass over jp = 0 .. Np - 1).  GT: the tables
// are read from global memory, as in k_interp_up_chunked.
template <typename T, int JM, bool GT>
__global__ void __launch_bounds__(256) k_anterp_dn_chunked(int Kc, int Lc, int Kp, int Lp, int nrhs, int cw_max,
                                                  const int *__restrict__ parent, const int *__restrict__ oct,
                                                  const T *__restrict__ tpc, const T *__restrict__ tpp,
                                                  const T *__restrict__ Phi, const T *__restrict__ Thp,
                                                  const T *__restrict__ Thm, const cx<T> *__restrict__ dn,
                                                  const cx<T> *__restrict__ Ip, cx<T> *__restrict__ Ic) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int Q = 3 * JM, IC = 2;
  const int Nc = 2 * Lc + 2, Np = 2 * Lp + 2, nthc = Lc + 1, nthp = Lp + 1, hp = Lp + 1, hc = Lc + 1;
  const int CW = cw_max, G2 = 2 * cw_max;
  cx<T> *A = reinterpret_cast<cx<T> *>(smem_raw);  // [Q][nthp][2 CW]: parent columns (jp, jp + hp) at (jl, CW + jl)
  cx<T> *G = A + (size_t)Q * nthp * G2;             // [Q][nthc][2 CW]
  T *Ps = reinterpret_cast<T *>(G + (size_t)Q * nthc * G2);  // Phi [Np][Nc]
  T *Tps = Ps + Np * Nc, *Tms = Tps + nthp * nthc;           // [nthp][nthc]
  const int c = blockIdx.x, r = blockIdx.y, pb = parent[c], o = oct[c], tid = threadIdx.x, NT = blockDim.x;
  if (!GT) {
    for (int i = tid; i < Np * Nc; i += NT) Ps[i] = Phi[i];
    for (int i = tid; i < nthp * nthc; i += NT) {
      Tps[i] = Thp[i];
      Tms[i] = Thm[i];
    }
  }
  const T *Psa = GT ? Phi : Ps, *Tpa = GT ? Thp : Tps, *Tma = GT ? Thm : Tms;
  const int nicb = (nthc + IC - 1) / IC;
  // with gridDim.z = 2 each CTA takes one of the sources (J, M), else both in turn
  const int jm_beg = gridDim.z > 1 ? (int)blockIdx.z * JM : 0, jm_end = gridDim.z > 1 ? jm_beg + JM : 2;
  for (int jm0 = jm_beg; jm0 < jm_end; jm0 += JM) {
    for (int j0 = 0; j0 < hp; j0 += CW) {
      const int cw = min(CW, hp - j0);
      __syncthreads();  // A and G free again
      const int per_m = nthp * 2 * cw;
      for (int i = tid; i < JM * per_m; i += NT) {
        const int m = i / per_m, rem = i - m * per_m;
        int t, a;  // parent direction, index within the component's [nthp][2 CW] block
        if (cw == hp) {  // one chunk: the block is the parent sampling itself
          t = rem;
          a = rem;
        } else {
          const int ip = rem / (2 * cw), jj = rem - ip * (2 * cw);
          const int half = jj >= cw ? 1 : 0, jl = jj - half * cw;
          t = ip * Np + j0 + jl + half * hp;
          a = ip * G2 + half * CW + jl;
        }
        const cx<T> *it = Ip + (((size_t)pb * 4 + (jm0 + m) * 2) * nrhs + r) * Kp;
        const cx<T> sh = dn[(size_t)o * Kp + t];
        const cx<T> ut = sh * it[t], up_ = sh * it[(size_t)nrhs * Kp + t];
        const T *u = tpp + 6 * (size_t)t;
#pragma unroll
        for (int x = 0; x < 3; ++x) A[(size_t)(m * 3 + x) * nthp * G2 + a] = ut * u[x] + up_ * u[3 + x];
      }
      __syncthreads();
      // transpose of the theta step: G[q][ic][j] = sum_ip Th+[ip][ic] A[q][ip][j] + Th-[ip][ic] A[q][ip][j + Np/2]
      for (int task = tid; task < nicb * cw; task += NT) {
        const int cb = task / cw, jl = task - cb * cw, ic0 = cb * IC;
        cx<T> g0[IC][Q], g1[IC][Q];
        for (int ip = 0; ip < nthp; ++ip) {
          cx<T> aa[Q], ab[Q];
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            aa[q] = A[((size_t)q * nthp + ip) * G2 + jl];
            ab[q] = A[((size_t)q * nthp + ip) * G2 + CW + jl];
          }
#pragma unroll
          for (int k = 0; k < IC; ++k) {
            const int ic = min(ic0 + k, nthc - 1);
            const T w1 = Tpa[ip * nthc + ic], w2 = Tma[ip * nthc + ic];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
              g0[k][q].re = fma(w1, aa[q].re, fma(w2, ab[q].re, g0[k][q].re));
              g0[k][q].im = fma(w1, aa[q].im, fma(w2, ab[q].im, g0[k][q].im));
              g1[k][q].re = fma(w1, ab[q].re, fma(w2, aa[q].re, g1[k][q].re));
              g1[k][q].im = fma(w1, ab[q].im, fma(w2, aa[q].im, g1[k][q].im));
            }
          }
        }
#pragma unroll
        for (int k = 0; k < IC; ++k) {
          const int ic = ic0 + k;
          if (ic >= nthc) break;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            G[((size_t)q * nthc + ic) * G2 + jl] = g0[k][q];
            G[((size_t)q * nthc + ic) * G2 + CW + jl] = g1[k][q];
          }
        }
      }
      __syncthreads();
      // transpose of the phi step over this chunk's columns, projection to
      // (theta, phi) at the child directions, added into the child
      for (int task = tid; task < nthc * hc; task += NT) {
        const int ic = task / hc, jc = task - ic * hc;
        cx<T> c0[Q], c1[Q];
        // G columns jj: jp = j0 + jj for jj < cw, j0 + jj - cw + hp after (one chunk: jp = jj)
        for (int jj = 0; jj < 2 * cw; ++jj) {
          const int jp = j0 + (jj < cw ? jj : jj - cw + hp), gj = jj < cw ? jj : jj - cw + CW;
          const T f0 = Psa[jp * Nc + jc], f1 = Psa[jp * Nc + jc + hc];
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const cx<T> g = G[((size_t)q * nthc + ic) * G2 + gj];
            c0[q].re = fma(f0, g.re, c0[q].re);
            c0[q].im = fma(f0, g.im, c0[q].im);
            c1[q].re = fma(f1, g.re, c1[q].re);
            c1[q].im = fma(f1, g.im, c1[q].im);
          }
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int tc = ic * Nc + jc + half * hc;
          const T *u = tpc + 6 * (size_t)tc;
#pragma unroll
          for (int m = 0; m < JM; ++m) {
            const cx<T> *C = half ? &c1[3 * m] : &c0[3 * m];
            cx<T> *it = Ic + (((size_t)c * 4 + (jm0 + m) * 2) * nrhs + r) * Kc;
            it[tc] += C[0] * u[0] + C[1] * u[1] + C[2] * u[2];
            it[(size_t)nrhs * Kc + tc] += C[0] * u[3] + C[1] * u[4] + C[2] * u[5];
          }
        }
      }
    }
  }
}

// Diagonal M2L translation: I_b(k) = sum_{b' in IL(b)} T_{b-b'}(k) S_b'(k), 4 components.
// One warp per (target box, slice of 32 directions), the boxes fastest in the
// grid, so the CTAs in flight at one time share a slice of the translators.
template <typename T>
__global__ void __launch_bounds__(32) k_m2l(int nbox, int K, int nrhs, const int *__restrict__ il_ptr,
                                            const int *__restrict__ il_src, const int *__restrict__ il_slot,
                                            const cx<T> *__restrict__ Tr, const cx<T> *__restrict__ S,
                                            cx<T> *__restrict__ I) {
  int k = blockIdx.y * 32 + threadIdx.x;
  int b = blockIdx.x;
  if (k >= K) return;
  int e0 = il_ptr[b], e1 = il_ptr[b + 1];
  const size_t cs = (size_t)nrhs * K;  // component stride
  for (int r = 0; r < nrhs; ++r) {
    cx<T> a0, a1, a2, a3;
    int e = e0;
    // four interaction-list sources in flight per thread
    for (; e + 4 <= e1; e += 4) {
      int s[4], sl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        s[u] = __ldg(il_src + e + u);
        sl[u] = __ldg(il_slot + e + u);
      }
      cx<T> t[4], v[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        t[u] = Tr[(size_t)sl[u] * K + k];
        const cx<T> *src = S + ((size_t)s[u] * 4 * nrhs + r) * K + k;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[u][q] = src[q * cs];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a0 = cfma(t[u], v[u][0], a0);
        a1 = cfma(t[u], v[u][1], a1);
        a2 = cfma(t[u], v[u][2], a2);
        a3 = cfma(t[u], v[u][3], a3);
      }
    }
    for (; e < e1; ++e) {
      int s = il_src[e];
      cx<T> t = Tr[(size_t)il_slot[e] * K + k];
      const cx<T> *src = S + ((size_t)s * 4 * nrhs + r) * K + k;
      a0 = cfma(t, src[0], a0);
      a1 = cfma(t, src[cs], a1);
      a2 = cfma(t, src[2 * cs], a2);
      a3 = cfma(t, src[3 * cs], a3);
    }
    cx<T> *o = I + ((size_t)b * 4 * nrhs + r) * K + k;
    o[0] = a0;
    o[cs] = a1;
    o[2 * cs] = a2;
    o[3 * cs] = a3;
  }
}

// Diagonal M2L by sibling groups: the children of one box share most of their
// interaction lists, so one CTA takes a group (up to 8 targets) for a chunk of
// directions, thread k.  For each source of the union (entries staged in shared
// memory) the four S components are read once and applied to every member
// that has the source in its list, with that member's translator:
//   I_u(k) = sum_{sources s of u} T_{u-s}(k) S_s(k).
// Per source and direction: 4 pattern loads plus one translator load per
// member, instead of 4 + 1 per member and source.
template <typename T>
__global__ void __launch_bounds__(128) k_m2l_group(int K, int nrhs, const int *__restrict__ grp_ptr,
                                                  const int *__restrict__ grp_box, const int *__restrict__ grp_ent,
                                                  const cx<T> *__restrict__ Tr, const cx<T> *__restrict__ S,
                                                  cx<T> *__restrict__ I) {
  extern __shared__ __align__(16) int ents[];  // [n][10]
  const int g = blockIdx.y, r = blockIdx.z;
  const int e0 = grp_ptr[g], ne = grp_ptr[g + 1] - e0;
  for (int i = threadIdx.x; i < ne * 10; i += blockDim.x) ents[i] = grp_ent[(size_t)e0 * 10 + i];
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const size_t cs = (size_t)nrhs * K;
  cx<T> acc[8][4];
#pragma unroll 2
  for (int e = 0; e < ne; ++e) {
    const int *E = ents + 10 * e;
    const int src = E[0], mask = E[1];
    const cx<T> *sp = S + ((size_t)src * 4 * nrhs + r) * K + k;
    const cx<T> s0 = sp[0], s1 = sp[cs], s2 = sp[2 * cs], s3 = sp[3 * cs];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (mask & (1 << u)) {
        const cx<T> t = Tr[(size_t)E[2 + u] * K + k];
        acc[u][0] = cfma(t, s0, acc[u][0]);
        acc[u][1] = cfma(t, s1, acc[u][1]);
        acc[u][2] = cfma(t, s2, acc[u][2]);
        acc[u][3] = cfma(t, s3, acc[u][3]);
      }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int b = grp_box[8 * (size_t)g + u];
    if (b < 0) continue;
    cx<T> *o = I + ((size_t)b * 4 * nrhs + r) * K + k;
    o[0] = acc[u][0];
    o[cs] = acc[u][1];
    o[2 * cs] = acc[u][2];
    o[3 * cs] = acc[u][3];
  }
}

// Diagonal M2L by sibling groups, with the group's union list split over the
// SW warps of the CTA for one slice of 32 directions (lane = direction): warp
// w takes entries w, w + SW, ...; each keeps partial sums for all (up to 8)
// members; the warps' partials are then added in warp order (deterministic)
// and written.  Same loads per source as k_m2l_group (4 pattern values, one
// translator per member that has the source), with SW times more warps in
// flight per direction slice, which a single right-hand side needs to fill the GPU.
template <typename T, int SW>
__global__ void __launch_bounds__(32 * SW) k_m2l_split(int K, int nrhs, const int *__restrict__ grp_ptr,
                                                      const int *__restrict__ grp_box, const int *__restrict__ grp_ent,
                                                      const cx<T> *__restrict__ Tr, const cx<T> *__restrict__ S,
                                                      cx<T> *__restrict__ I) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T> *part = reinterpret_cast<cx<T> *>(smem_raw);                 // [SW - 1][8][4][32]
  int *ents = reinterpret_cast<int *>(part + (size_t)(SW - 1) * 8 * 4 * 32);  // [n][10]
  const int g = blockIdx.y, r = blockIdx.z, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e0 = grp_ptr[g], ne = grp_ptr[g + 1] - e0;
  for (int i = threadIdx.x; i < ne * 10; i += blockDim.x) ents[i] = grp_ent[(size_t)e0 * 10 + i];
  __syncthreads();
  const int k = blockIdx.x * 32 + lane;
  const bool kin = k < K;
  const int kk = kin ? k : K - 1;  // out-of-range lanes load a valid direction, write nothing
  const size_t cs = (size_t)nrhs * K;
  cx<T> acc[8][4];
  for (int e = warp; e < ne; e += SW) {
    const int *E = ents + 10 * e;
    const int src = E[0], mask = E[1];
    const cx<T> *sp = S + ((size_t)src * 4 * nrhs + r) * K + kk;
    const cx<T> s0 = sp[0], s1 = sp[cs], s2 = sp[2 * cs], s3 = sp[3 * cs];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (mask & (1 << u)) {
        const cx<T> t = Tr[(size_t)E[2 + u] * K + kk];
        acc[u][0] = cfma(t, s0, acc[u][0]);
        acc[u][1] = cfma(t, s1, acc[u][1]);
        acc[u][2] = cfma(t, s2, acc[u][2]);
        acc[u][3] = cfma(t, s3, acc[u][3]);
      }
  }
  if (warp > 0) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) part[(((size_t)(warp - 1) * 8 + u) * 4 + q) * 32 + lane] = acc[u][q];
  }
  __syncthreads();
  if (warp != 0 || !kin) return;
#pragma unroll
  for (int w = 1; w < SW; ++w)
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[u][q] += part[(((size_t)(w - 1) * 8 + u) * 4 + q) * 32 + lane];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int b = grp_box[8 * (size_t)g + u];
    if (b < 0) continue;
    cx<T> *o = I + ((size_t)b * 4 * nrhs + r) * K + k;
    o[0] = acc[u][0];
    o[cs] = acc[u][1];
    o[2 * cs] = acc[u][2];
    o[3 * cs] = acc[u][3];
  }
}

// Leaf receive with the JMCFIE weights of medium l (weights and constants
// folded into the translators).  Per box the combined fields
//   F1 = I^J - khat x I^M / eta,   F3 = -eta khat x I^J - I^M,
// khat x (a_t, a_p) = (-a_p, a_t), are formed once in shared memory; then each
// basis (one warp, lanes over k) takes
//   y_J += sum_k P_t F1_t + P_p F1_p,   y_M -= sum_k P_t F3_t + P_p F3_p
// with its combined receive pattern P (antipodal radiation pattern for the
// tangential test, t x n pattern for the n x operators, signs folded in).
// The box's P block streams through shared memory as in k_aggregate.
// The sums are formed in T and added into y of type TY (FP32 far field into
// an FP64 product for the true residual of the mixed form).
template <typename T, int RB, typename TY>
__global__ void __launch_bounds__(256) k_disaggregate(int K, int ne, int nrhs, int cb,
                                                     const int *__restrict__ box_start,
                                                     const int *__restrict__ basis_p, const cx<T> *__restrict__ P,
                                                     const cx<T> *__restrict__ I, cx<T> eta, cx<T> ieta,
                                                     cx<TY> *__restrict__ y, cx<T> cJ, cx<T> cM,
                                                     cx<T> *__restrict__ part, int part_off, int part_nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x, i0 = box_start[b], n = box_start[b + 1] - i0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const size_t per = (size_t)2 * K;
  cx<T> *ring = reinterpret_cast<cx<T> *>(smem_raw);  // [STAGES][cb][2][K]
  cx<T> *F = ring + (size_t)STAGES * cb * per;        // [RB][4][K]: F1t, F1p, F3t, F3p
  const size_t cs = (size_t)nrhs * K;
  const int nch = (n + cb - 1) / cb;
  auto fetch = [&](int ch) {
    if (ch < nch) {
      const int li0 = ch * cb, m = min(cb, n - li0);
      cta_copy_async(ring + (size_t)(ch % STAGES) * cb * per, P + (size_t)(i0 + li0) * per,
                     (size_t)m * per * sizeof(cx<T>));
    }
    cp_async_commit_s();
  };
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int nr = min(RB, nrhs - r0);
    for (int ch = 0; ch < STAGES; ++ch) fetch(ch);
    for (int idx = threadIdx.x; idx < nr * K; idx += blockDim.x) {
      const int rr = idx / K, k = idx - rr * K;
      const cx<T> *Ib = I + ((size_t)b * 4 * nrhs + r0 + rr) * K + k;
      const cx<T> iJt = Ib[0], iJp = Ib[cs], iMt = Ib[2 * cs], iMp = Ib[3 * cs];
      cx<T> *f = F + (size_t)rr * 4 * K + k;
      f[0] = iJt + iMp * ieta;
      f[K] = iJp - iMt * ieta;
      f[2 * K] = eta * iJp - iMt;
      f[3 * K] = -(eta * iJt) - iMp;
    }
    for (int ch = 0; ch < nch; ++ch) {
      cp_async_wait_s<STAGES - 1>();
      __syncthreads();  // chunk ch (and, the first time, the fields) visible to all
      const int li0 = ch * cb, m = min(cb, n - li0);
      const cx<T> *pc = ring + (size_t)(ch % STAGES) * cb * per;
      for (int li = warp; li < m; li += nw) {
        const cx<T> *Pi = pc + (size_t)li * per;
        cx<T> yj[RB], ym[RB];
        for (int k = lane; k < K; k += 32) {
          const cx<T> pt = Pi[k], pp = Pi[K + k];
#pragma unroll
          for (int rr = 0; rr < RB; ++rr)
            if (rr < nr) {
              const cx<T> *f = F + (size_t)rr * 4 * K + k;
              yj[rr] = cfma(pt, f[0], cfma(pp, f[K], yj[rr]));
              ym[rr] = cfma(pt, f[2 * K], cfma(pp, f[3 * K], ym[rr]));
            }
        }
        const int p = basis_p[i0 + li0 + li];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
          if (rr < nr) {
            const cx<T> sj = warp_sum(yj[rr]), sm = warp_sum(ym[rr]);
            if (lane == 0) {
              if (part) {  // this medium's rows, added into y later in medium order
                cx<T> *o = part + ((size_t)(r0 + rr) * part_nb + part_off + i0 + li0 + li) * 2;
                o[0] = cJ * sj;
                o[1] = cM * sm;
              } else {
                cx<TY> *o = y + ((size_t)(r0 + rr) * ne + p) * 2;
                o[0] += cx<TY>(cJ * sj);
                o[1] -= cx<TY>(cM * sm);
              }
            }
          }
      }
      __syncthreads();  // the stage is free again
      fetch(ch + STAGES);
    }
    cp_async_wait_s<0>();
    __syncthreads();
  }
}

// The receives' rows added into y in medium order (the lower medium first, as
// when the receives add into y one medium after another):
//   y_J += r_J(a) + ... ,  y_M -= r_M(a) ... ; thread = (right-hand side, basis).
template <typename T, typename TY>
__global__ void k_rec_combine(int ne, int nrhs, int part_nb, const int *__restrict__ rmap,
                              const cx<T> *__restrict__ part, cx<TY> *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nrhs * ne) return;
  const int r = (int)(i / ne), p = (int)(i - (int64_t)r * ne);
  cx<TY> *o = y + i * 2;
  cx<TY> yj = o[0], ym = o[1];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int a = rmap[2 * (size_t)p + j];
    if (a < 0) continue;
    const cx<T> *q = part + ((size_t)r * part_nb + a) * 2;
    yj += cx<TY>(q[0]);
    ym -= cx<TY>(q[1]);
  }
  o[0] = yj;
  o[1] = ym;
}

// ---------------------------------------------------------------- ILU(0) sweeps
// The factors are stored in the box-colour order: for colour c, the rows of
// all its leaf boxes are contiguous and no two of its boxes touch, so a box's
// rows couple only to its own rows and to rows of other colours.  One launch
// per colour and sweep, one CTA per box of the colour:
//   (1) t_b = src_b - sum_q F_bq z_q over the off-box blocks of the box's rows
//       (earlier colours in the forward sweep, later ones in the backward);
//   (2) z_b = L_bb^{-1} t_b (forward) or U_bb^{-1} t_b (backward).
// The in-box inverses are formed once at setup, so (2) is a dense product
// instead of a sequential substitution; z equals the substitution result up
// to rounding.  The inverses are packed by rows: forward, row i holds the
// blocks j < i of L_bb^{-1} (its diagonal blocks are identities); backward,
// row i holds the blocks j >= i of U_bb^{-1}.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ cx<T> shfl_up(cx<T> v, int d) {
  return cx<T>(__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d));
}

// Single right-hand side: the off-box products are pushed one source colour
// at a time, so that each launch has the whole GPU's worth of short rows.
// Sweep step for colour c with source colour sc (forward: c-1, backward: c+1):
//   role A, the boxes B of colour c (one CTA per piece, below):
//       t_B = w_B - F_{B,sc} z_sc,   z_B = L_BB^{-1} t_B   (U_BB^{-1} backward);
//       the last forward step also applies U_BB^{-1} (colour 7 has no later colour);
//   role B, ILU_RL lanes per row i of the colours still to come:
//       w_i -= F_{i,sc} z_sc   (the first forward step copies w = src).
// w lives in z until the row is solved.  Each row's off-box blocks are sorted
// by column, hence grouped by colour; cptr[i][c] .. cptr[i][c+1] is colour c.
// In role A the box's blocks from sc (its "virtual range") are cut into
// pieces of at most 1024 blocks (cut at setup), one CTA per piece, so that a large box
// does not hold up the launch.  Within a piece the blocks are spread evenly over the CTA in
// groups of 32 (one per lane); a segmented scan over the lanes keyed by row
// adds each row's products, every warp keeps its own row partials, and the
// warps' partials are added in warp order.  A box of one piece finishes in its
// CTA, with its packed in-box inverse copied to shared memory asynchronously
// meanwhile.  A box of several pieces: each piece writes its row partials to
// scratch and counts itself in; the last to arrive adds the pieces' partials
// in piece order and finishes the box.  The results are deterministic.
// The sweep steps are chained (programmatic dependent launch, common.h): a
// step reads its static prologue (row colour pointers, prefixes, the packed
// inverse) while the previous step drains, and waits before it touches z.

constexpr int ILU_RL = 8;  // lanes per pushed row
constexpr int ILU_RU = 2;  // blocks per lane and iteration of a pushed row

// One work item of a sweep step: a piece of a box of the step's colour
// (role A, item < npieceA) or a group of rows of the colours still to come
// (role B).  CHAINED: launched as its own grid with programmatic dependent
// launch (static prologue before pdl_wait); otherwise called from the
// persistent kernel, where a grid barrier separates the steps.  Values written
// earlier in the same launch (z, w, the piece partials) are read through L2
// (ld.global.cg): L1 is not coherent across CTAs within a launch.
template <typename T, int NT, bool CHAINED>
__device__ __forceinline__ void ilu_item(int item, int forward, int both, int colour, int npieceA,
                                         const int *__restrict__ pieces, int rb0, int rb1, int stage_tri, int nmax,
                                         cx<T> *scratch, int *counter, const int *__restrict__ box_start,
                                         const int *__restrict__ cptr, const int *__restrict__ off_col,
                                         const cx<T> *__restrict__ off_val, const int64_t *__restrict__ tri_off,
                                         const cx<T> *__restrict__ tri, const int64_t *__restrict__ tri2_off,
                                         const cx<T> *__restrict__ tri2, const cx<T> *src, cx<T> *z,
                                         unsigned char *smem_raw) {
  constexpr int NW = NT / 32;
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V16;
  constexpr int NV = (int)(4 * sizeof(cx<T>) / sizeof(V16));
  const V16 *Ov = reinterpret_cast<const V16 *>(off_val);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sc = forward ? colour - 1 : colour + 1;
  const bool has_src = sc >= 0 && sc < 8;
  // w of rows not yet solved: src before the first forward step has run
  const cx<T> *w = (forward && colour == 0) ? src : z;
  if (item >= npieceA) {
    // ---- role B: rows of later colours take the contribution of colour sc;
    // ILU_RL lanes per row (rows hold about 40 blocks per source colour)
    const int hl = lane & (ILU_RL - 1);
    const int i = rb0 + (item - npieceA) * (32 / ILU_RL) * NW + (32 / ILU_RL) * warp + lane / ILU_RL;
    const bool row_ok = i < rb1;
    int q0 = 0, q1 = 0;
    if (row_ok && has_src) {
      q0 = cptr[9 * (size_t)i + sc];
      q1 = cptr[9 * (size_t)i + sc + 1];
    }
    if (CHAINED) {
      pdl_wait();
      pdl_release();
    }
    if (!has_src) {
      if (row_ok && hl < 2) z[2 * (size_t)i + hl] = src[2 * (size_t)i + hl];
      return;
    }
    cx<T> a0, a1;
    int q = q0 + hl;
    // ILU_RU blocks per lane and iteration: their column and value loads are
    // issued together, then the z gathers they select
    for (; q + (ILU_RU - 1) * ILU_RL < q1; q += ILU_RU * ILU_RL) {
      int cc[ILU_RU];
      V16 uu[ILU_RU][NV];
#pragma unroll
      for (int u = 0; u < ILU_RU; ++u) {
        cc[u] = __ldg(off_col + q + u * ILU_RL);
#pragma unroll
        for (int v = 0; v < NV; ++v) uu[u][v] = __ldg(Ov + (size_t)(q + u * ILU_RL) * NV + v);
      }
      cx<T> xx[ILU_RU][2];
#pragma unroll
      for (int u = 0; u < ILU_RU; ++u) ldz_pair<CHAINED>(z + 2 * (size_t)cc[u], xx[u][0], xx[u][1]);
#pragma unroll
      for (int u = 0; u < ILU_RU; ++u) {
        const cx<T> *bb = reinterpret_cast<const cx<T> *>(uu[u]);
        a0 = cfma(bb[0], xx[u][0], cfma(bb[1], xx[u][1], a0));
        a1 = cfma(bb[2], xx[u][0], cfma(bb[3], xx[u][1], a1));
      }
    }
    for (; q < q1; q += ILU_RL) {
      const int c0 = __ldg(off_col + q);
      V16 u0[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u0[v] = __ldg(Ov + (size_t)q * NV + v);
      cx<T> x0, x1;
      ldz_pair<CHAINED>(z + 2 * (size_t)c0, x0, x1);
      const cx<T> *b0 = reinterpret_cast<const cx<T> *>(u0);
      a0 = cfma(b0[0], x0, cfma(b0[1], x1, a0));
      a1 = cfma(b0[2], x0, cfma(b0[3], x1, a1));
    }
#pragma unroll
    for (int d = ILU_RL / 2; d > 0; d >>= 1) {  // within the row's lanes
      a0 += shfl_down(a0, d);
      a1 += shfl_down(a1, d);
    }
    if (row_ok && hl == 0 && q1 > q0) {
      z[2 * (size_t)i] = ldcg_cx(z + 2 * (size_t)i) - a0;
      z[2 * (size_t)i + 1] = ldcg_cx(z + 2 * (size_t)i + 1) - a1;
    }
    return;
  }
  // ---- role A: one piece of a box of this colour
  const int *pc = pieces + 5 * (size_t)item;
  const int b = pc[0], v0 = pc[1], v1 = pc[2], kp = pc[3], np = pc[4];
  const int s0 = box_start[b], n = box_start[b + 1] - s0;
  const int ntri = forward ? n * (n - 1) / 2 : n * (n + 1) / 2;
  const cx<T> *Mg = tri + 4 * tri_off[b];
  stage_tri = stage_tri && np == 1;  // only a box that finishes in this CTA prefetches its inverse
  // shared: [packed triangle (if staged)] [NW][n][2] partials, [2n] t, [2n] t2, [n+1] prefix, [n] starts
  cx<T> *Ms = reinterpret_cast<cx<T> *>(smem_raw);
  cx<T> *part = Ms + (stage_tri ? 4 * (size_t)ntri : 0);
  cx<T> *t = part + (size_t)NW * 2 * n;
  cx<T> *t2 = t + 2 * n;
  int *pre = reinterpret_cast<int *>(t2 + 2 * n);
  int *st = pre + n + 1;
  if (stage_tri) {
    const size_t bytes = (size_t)ntri * 4 * sizeof(cx<T>);
    const char *g = reinterpret_cast<const char *>(Mg);
    char *d = reinterpret_cast<char *>(Ms);
    for (size_t o = (size_t)threadIdx.x * 16; o < bytes; o += (size_t)NT * 16) cp_async16(d + o, g + o);
    cp_async_commit();
  }
  for (int idx = threadIdx.x; idx < NW * 2 * n; idx += NT) part[idx] = cx<T>();
  if (warp == 0) {
    // prefix of the rows' block counts from colour sc
    int carry = 0;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int li = c0 + lane;
      int len = 0;
      if (li < n && has_src) {
        const int a = cptr[9 * (size_t)(s0 + li) + sc];
        len = cptr[9 * (size_t)(s0 + li) + sc + 1] - a;
        st[li] = a;
      }
      int inc = len;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
      }
      if (li < n) pre[li] = carry + inc - len;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) pre[n] = carry;
  }
  __syncthreads();
  if (CHAINED) {
    pdl_wait();  // z, w and the piece scratch below come from earlier steps
    pdl_release();
  }
  const int total = v1;  // this piece: virtual indices [v0, v1) of the box's blocks from sc
  const int ng = (v1 - v0 + 31) >> 5;
  const int g0 = (int)((int64_t)warp * ng / NW), g1 = (int)((int64_t)(warp + 1) * ng / NW);
  cx<T> *pw = part + (size_t)warp * 2 * n;
  // virtual index v of the box's blocks -> row (last row whose prefix is <= v) and block index
  auto locate = [&](int v, int &r, int &q) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= v) lo = mid;
      else hi = mid - 1;
    }
    r = lo;
    q = st[lo] + v - pre[lo];
  };
  auto segsum = [&](int r, cx<T> p0, cx<T> p1) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const cx<T> u0 = shfl_up(p0, d), u1 = shfl_up(p1, d);
      const int ru = __shfl_up_sync(0xffffffffu, r, d);
      if (lane >= d && ru == r) {
        p0 += u0;
        p1 += u1;
      }
    }
    const int rn = __shfl_down_sync(0xffffffffu, r, 1);
    if (r >= 0 && (lane == 31 || rn != r)) {
      pw[2 * r] += p0;
      pw[2 * r + 1] += p1;
    }
    __syncwarp();
  };
  for (int g = g0; g < g1; g += 2) {
    // two groups in flight: issue both groups' loads, then reduce
    const int vA = v0 + g * 32 + lane, vB = vA + 32;
    const bool hasB = g + 1 < g1;
    int rA = -1, rB = -1, qA = 0, qB = 0, cA = 0, cB = 0;
    V16 uA[NV], uB[NV];
    if (vA < total) {
      locate(vA, rA, qA);
      cA = __ldg(off_col + qA);
#pragma unroll
      for (int v = 0; v < NV; ++v) uA[v] = __ldg(Ov + (size_t)qA * NV + v);
    }
    if (hasB && vB < total) {
      locate(vB, rB, qB);
      cB = __ldg(off_col + qB);
#pragma unroll
      for (int v = 0; v < NV; ++v) uB[v] = __ldg(Ov + (size_t)qB * NV + v);
    }
    cx<T> a0, a1, b0, b1;
    if (rA >= 0) {
      const cx<T> *bb = reinterpret_cast<const cx<T> *>(uA);
      cx<T> x0, x1;
      ldz_pair<CHAINED>(z + 2 * (size_t)cA, x0, x1);
      a0 = cfma(bb[0], x0, bb[1] * x1);
      a1 = cfma(bb[2], x0, bb[3] * x1);
    }
    if (rB >= 0) {
      const cx<T> *bb = reinterpret_cast<const cx<T> *>(uB);
      cx<T> x0, x1;
      ldz_pair<CHAINED>(z + 2 * (size_t)cB, x0, x1);
      b0 = cfma(bb[0], x0, bb[1] * x1);
      b1 = cfma(bb[2], x0, bb[3] * x1);
    }
    segsum(rA, a0, a1);
    if (hasB) segsum(rB, b0, b1);
  }
  __syncthreads();
  if (np == 1) {
    for (int li = threadIdx.x; li < n; li += NT) {
      cx<T> u0 = ldcg_cx(w + 2 * (size_t)(s0 + li)), u1 = ldcg_cx(w + 2 * (size_t)(s0 + li) + 1);
      for (int ww = 0; ww < NW; ++ww) {
        u0 -= part[(size_t)ww * 2 * n + 2 * li];
        u1 -= part[(size_t)ww * 2 * n + 2 * li + 1];
      }
      t[2 * li] = u0;
      t[2 * li + 1] = u1;
    }
  } else {
    cx<T> *mine = scratch + (size_t)item * 2 * nmax;
    for (int li = threadIdx.x; li < n; li += NT) {
      cx<T> u0, u1;
      for (int ww = 0; ww < NW; ++ww) {
        u0 += part[(size_t)ww * 2 * n + 2 * li];
        u1 += part[(size_t)ww * 2 * n + 2 * li + 1];
      }
      mine[2 * li] = u0;
      mine[2 * li + 1] = u1;
    }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) s_last = atomicAdd(&counter[b], 1) == np - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) counter[b] = 0;  // ready for the next launch
    const cx<T> *first = scratch + (size_t)(item - kp) * 2 * nmax;
    for (int li = threadIdx.x; li < n; li += NT) {
      cx<T> u0 = ldcg_cx(w + 2 * (size_t)(s0 + li)), u1 = ldcg_cx(w + 2 * (size_t)(s0 + li) + 1);
      for (int k = 0; k < np; ++k) {
        const cx<T> *pk = first + (size_t)k * 2 * nmax + 2 * li;
        u0 -= ldcg_cx(pk);
        u1 -= ldcg_cx(pk + 1);
      }
      t[2 * li] = u0;
      t[2 * li + 1] = u1;
    }
  }
  if (stage_tri) cp_async_wait_all();
  __syncthreads();
  // in-box product(s): rows one per warp, lanes over the row's packed blocks
  for (int pass = 0; pass < (both ? 2 : 1); ++pass) {
    const bool lower = forward && pass == 0;
    const cx<T> *M = pass == 0 ? (stage_tri ? Ms : Mg) : tri2 + 4 * tri2_off[b];
    const cx<T> *in = pass == 0 ? t : t2;
    for (int li = warp; li < n; li += NW) {
      const int j0 = lower ? 0 : li, j1 = lower ? li : n;
      const cx<T> *row = M + 4 * (size_t)(lower ? li * (li - 1) / 2 : li * n - li * (li - 1) / 2);
      cx<T> a0, a1;
      for (int j = j0 + lane; j < j1; j += 32) {
        const cx<T> *B = row + 4 * (j - j0);
        const cx<T> x0 = in[2 * j], x1 = in[2 * j + 1];
        a0 = cfma(B[0], x0, cfma(B[1], x1, a0));
        a1 = cfma(B[2], x0, cfma(B[3], x1, a1));
      }
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      if (lane == 0) {
        if (lower) {
          a0 += in[2 * li];
          a1 += in[2 * li + 1];
        }
        if (both && pass == 0) {
          t2[2 * li] = a0;
          t2[2 * li + 1] = a1;
        } else {
          z[2 * (size_t)(s0 + li)] = a0;
          z[2 * (size_t)(s0 + li) + 1] = a1;
        }
      }
    }
    if (both && pass == 0) __syncthreads();
  }
}


template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_ilu_sweep(int forward, int both, int colour, int npieceA,
                                                  const int *__restrict__ pieces, int rb0, int rb1, int stage_tri,
                                                  int nmax, cx<T> *scratch, int *counter,
                                                  const int *__restrict__ box_start,
                                                  const int *__restrict__ cptr, const int *__restrict__ off_col,
                                                  const cx<T> *__restrict__ off_val,
                                                  const int64_t *__restrict__ tri_off, const cx<T> *__restrict__ tri,
                                                  const int64_t *__restrict__ tri2_off,
                                                  const cx<T> *__restrict__ tri2, const cx<T> *src, cx<T> *z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ilu_item<T, NT, true>((int)blockIdx.x, forward, both, colour, npieceA, pieces, rb0, rb1, stage_tri, nmax, scratch,
                        counter, box_start, cptr, off_col, off_val, tri_off, tri, tri2_off, tri2, src, z, smem_raw);
}

// The whole single-RHS apply in one cooperative launch: the 15 sweep steps run
// in order, each over all resident CTAs (work items taken in index order with
// a stride of the grid size), separated by a grid barrier: every CTA counts
// itself in on a device-scope counter (release) and waits (acquire) until the
// whole grid has arrived.  The wait is bounded: after wait_limit polls the
// CTA records SIE_ETIMEOUT's cause in *err and returns, and every other CTA
// gives up at its next barrier once *err is set, so the launch always ends.
// *bar must be zero at launch (cleared on the stream before it).
struct IluStepDesc {
  int forward, both, colour, npieceA, piece0, rb0, rb1, nitems;
  const int *cptr, *col;
  const void *val;
  const int64_t *tri_off;
  const void *tri;
};
struct IluPlan {
  IluStepDesc s[15];
  int nsteps;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// false when the wait gave up (limit reached, or another CTA gave up first)
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned target, int wait_limit, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    for (int it = 0;; ++it) {
      if (it >= wait_limit || *(volatile int *)err) {
        ok = 0;
        atomicOr(err, 1);
        break;
      }
      if (ld_acquire_gpu(bar) >= target) break;
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) k_ilu_persistent(IluPlan P, const int *__restrict__ pieces, int stage_tri,
                                                          int nmax, cx<T> *scratch, int *counter,
                                                          const int *__restrict__ box_start,
                                                          const int64_t *__restrict__ tu_off,
                                                          const cx<T> *__restrict__ tu, const cx<T> *src, cx<T> *z,
                                                          unsigned *bar, int wait_limit, int *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int st = 0; st < P.nsteps; ++st) {
    const IluStepDesc &S = P.s[st];
    for (int it = blockIdx.x; it < S.nitems; it += gridDim.x) {
      ilu_item<T, NT, false>(it, S.forward, S.both, S.colour, S.npieceA, pieces + 5 * (size_t)S.piece0, S.rb0, S.rb1,
                             stage_tri, nmax, scratch, counter, box_start, S.cptr, S.col,
                             reinterpret_cast<const cx<T> *>(S.val), S.tri_off, reinterpret_cast<const cx<T> *>(S.tri),
                             tu_off, tu, src, z, smem_raw);
      __syncthreads();  // shared memory is reused by the next item
    }
    if (st + 1 < P.nsteps && !grid_barrier(bar, (unsigned)(st + 1) * gridDim.x, wait_limit, err)) return;
  }
}

// Block of right-hand sides: the same 15 sweep steps as the single-RHS path,
// RB right-hand sides sharing every block load.  Role A: one CTA per box of
// the colour, rows one per warp over the row's blocks from the source colour,
// then the in-box inverse(s); role B: 8 lanes per row of the colours still to
// come.  Right-hand sides beyond RB are taken in further passes.
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_ilu_sweep_blk(int ne, int nrhs, int forward, int both, int colour,
                                                      int nboxA, int box0, int rb0, int rb1,
                                                      const int *__restrict__ box_start,
                                                      const int *__restrict__ cptr, const int *__restrict__ off_col,
                                                      const cx<T> *__restrict__ off_val,
                                                      const int64_t *__restrict__ tri_off,
                                                      const cx<T> *__restrict__ tri,
                                                      const int64_t *__restrict__ tri2_off,
                                                      const cx<T> *__restrict__ tri2, const cx<T> *src, cx<T> *z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V16;
  constexpr int NV = (int)(4 * sizeof(cx<T>) / sizeof(V16));
  const V16 *Ov = reinterpret_cast<const V16 *>(off_val);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const size_t vs = (size_t)ne * 2;
  const int sc = forward ? colour - 1 : colour + 1;
  const bool has_src = sc >= 0 && sc < 8;
  const cx<T> *w = (forward && colour == 0) ? src : z;
  if ((int)blockIdx.x >= nboxA) {
    // ---- role B
    const int hl = threadIdx.x & 7;
    const int i = rb0 + ((int)blockIdx.x - nboxA) * ((int)blockDim.x / 8) + (int)(threadIdx.x >> 3);
    const bool row_ok = i < rb1;
    if (!has_src) {
      if (row_ok)
        for (int rr = 0; rr < nrhs; ++rr)
          if (hl < 2) z[(size_t)rr * vs + 2 * (size_t)i + hl] = src[(size_t)rr * vs + 2 * (size_t)i + hl];
      return;
    }
    int q0 = 0, q1 = 0;
    if (row_ok) {
      q0 = cptr[9 * (size_t)i + sc];
      q1 = cptr[9 * (size_t)i + sc + 1];
    }
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
      const int nr = min(RB, nrhs - r0);
      cx<T> a0[RB], a1[RB];
      for (int q = q0 + hl; q < q1; q += 8) {
        const int cc = __ldg(off_col + q);
        V16 u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = __ldg(Ov + (size_t)q * NV + v);
        const cx<T> *bb = reinterpret_cast<const cx<T> *>(u);
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
          if (rr < nr) {
            cx<T> x0, x1;
            ldg_pair(z + (size_t)(r0 + rr) * vs + 2 * (size_t)cc, x0, x1);  // colour sc: not written here
            a0[rr] = cfma(bb[0], x0, cfma(bb[1], x1, a0[rr]));
            a1[rr] = cfma(bb[2], x0, cfma(bb[3], x1, a1[rr]));
          }
      }
#pragma unroll
      for (int rr = 0; rr < RB; ++rr) {
#pragma unroll
        for (int d = 4; d > 0; d >>= 1) {
          a0[rr] += shfl_down(a0[rr], d);
          a1[rr] += shfl_down(a1[rr], d);
        }
        if (rr < nr && row_ok && hl == 0 && q1 > q0) {
          cx<T> *o = z + (size_t)(r0 + rr) * vs + 2 * (size_t)i;
          o[0] -= a0[rr];
          o[1] -= a1[rr];
        }
      }
    }
    return;
  }
  // ---- role A
  cx<T> *t = reinterpret_cast<cx<T> *>(smem_raw);  // [RB][2n]
  const int b = box0 + blockIdx.x;
  const int s0 = box_start[b], n = box_start[b + 1] - s0;
  cx<T> *t2 = t + (size_t)RB * 2 * n;               // [RB][2n]
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int nr = min(RB, nrhs - r0);
    for (int li = warp; li < n; li += nw) {
      const int i = s0 + li;
      const int q0 = has_src ? cptr[9 * (size_t)i + sc] : 0, q1 = has_src ? cptr[9 * (size_t)i + sc + 1] : 0;
      cx<T> a0[RB], a1[RB];
      for (int q = q0 + lane; q < q1; q += 32) {
        const int cc = __ldg(off_col + q);
        V16 u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = __ldg(Ov + (size_t)q * NV + v);
        const cx<T> *bb = reinterpret_cast<const cx<T> *>(u);
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
          if (rr < nr) {
            cx<T> x0, x1;
            ldg_pair(z + (size_t)(r0 + rr) * vs + 2 * (size_t)cc, x0, x1);
            a0[rr] = cfma(bb[0], x0, cfma(bb[1], x1, a0[rr]));
            a1[rr] = cfma(bb[2], x0, cfma(bb[3], x1, a1[rr]));
          }
      }
#pragma unroll
      for (int rr = 0; rr < RB; ++rr)
        if (rr < nr) {
          const cx<T> u0 = warp_sum(a0[rr]), u1 = warp_sum(a1[rr]);
          if (lane == 0) {
            const cx<T> *wr = w + (size_t)(r0 + rr) * vs + 2 * (size_t)i;
            t[(size_t)rr * 2 * n + 2 * li] = wr[0] - u0;
            t[(size_t)rr * 2 * n + 2 * li + 1] = wr[1] - u1;
          }
        }
    }
    __syncthreads();
    for (int pass = 0; pass < (both ? 2 : 1); ++pass) {
      const bool lower = forward && pass == 0;
      const cx<T> *M = pass == 0 ? tri + 4 * tri_off[b] : tri2 + 4 * tri2_off[b];
      const cx<T> *in = pass == 0 ? t : t2;
      for (int li = warp; li < n; li += nw) {
        const int j0 = lower ? 0 : li, j1 = lower ? li : n;
        const cx<T> *row = M + 4 * (size_t)(lower ? li * (li - 1) / 2 : li * n - li * (li - 1) / 2);
        cx<T> a0[RB], a1[RB];
        for (int j = j0 + lane; j < j1; j += 32) {
          const cx<T> *B = row + 4 * (j - j0);
          const cx<T> b0 = B[0], b1 = B[1], b2 = B[2], b3 = B[3];
#pragma unroll
          for (int rr = 0; rr < RB; ++rr)
            if (rr < nr) {
              const cx<T> x0 = in[(size_t)rr * 2 * n + 2 * j], x1 = in[(size_t)rr * 2 * n + 2 * j + 1];
              a0[rr] = cfma(b0, x0, cfma(b1, x1, a0[rr]));
              a1[rr] = cfma(b2, x0, cfma(b3, x1, a1[rr]));
            }
        }
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
          if (rr < nr) {
            cx<T> u0 = warp_sum(a0[rr]), u1 = warp_sum(a1[rr]);
            if (lane == 0) {
              if (lower) {
                u0 += in[(size_t)rr * 2 * n + 2 * li];
                u1 += in[(size_t)rr * 2 * n + 2 * li + 1];
              }
              if (both && pass == 0) {
                t2[(size_t)rr * 2 * n + 2 * li] = u0;
                t2[(size_t)rr * 2 * n + 2 * li + 1] = u1;
              } else {
                cx<T> *o = z + (size_t)(r0 + rr) * vs + 2 * (size_t)(s0 + li);
                o[0] = u0;
                o[1] = u1;
              }
            }
          }
      }
      __syncthreads();
    }
  }
}

// The block sweeps on right-hand-side-interleaved vectors: zT[(2 i + c) Rp + r]
// (row i, J/M component c, right-hand side r < Rp, Rp a multiple of RB, the
// padding right-hand sides zero).  The same 15 steps and roles as
// k_ilu_sweep_blk, but the RB values of one vector entry are one contiguous,
// aligned run, so each block of a factor gathers them with RB / 2 (FP32) or
// RB (FP64) 16-byte loads instead of RB scattered ones; the padding lanes
// carry zeros through (the sweep is linear), so no lane is masked.
template <typename T, int RB>
__device__ __forceinline__ void ld_rb(const cx<T> *__restrict__ p, cx<T> (&x)[RB]) {
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V16;
  constexpr int PER = (int)(sizeof(V16) / sizeof(cx<T>));
  const V16 *q = reinterpret_cast<const V16 *>(p);
#pragma unroll
  for (int u = 0; u < RB / PER; ++u) {
    const V16 v = __ldcg(q + u);
    memcpy(&x[u * PER], &v, sizeof(V16));
  }
}

template <typename T, int RB>
__global__ void __launch_bounds__(256) k_ilu_sweep_blkT(int ne, int Rp, int forward, int both, int colour,
                                                       int nboxA, int box0, int rb0, int rb1,
                                                       const int *__restrict__ box_start,
                                                       const int *__restrict__ cptr,
                                                       const int *__restrict__ off_col,
                                                       const cx<T> *__restrict__ off_val,
                                                       const int64_t *__restrict__ tri_off,
                                                       const cx<T> *__restrict__ tri,
                                                       const int64_t *__restrict__ tri2_off,
                                                       const cx<T> *__restrict__ tri2, const cx<T> *src, cx<T> *z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V16;
  constexpr int NV = (int)(4 * sizeof(cx<T>) / sizeof(V16));
  const V16 *Ov = reinterpret_cast<const V16 *>(off_val);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int sc = forward ? colour - 1 : colour + 1;
  const bool has_src = sc >= 0 && sc < 8;
  const cx<T> *w = (forward && colour == 0) ? src : z;
  if ((int)blockIdx.x >= nboxA) {
    // ---- role B: 8 lanes per row of the colours still to come
    const int hl = threadIdx.x & 7;
    const int i = rb0 + ((int)blockIdx.x - nboxA) * ((int)blockDim.x / 8) + (int)(threadIdx.x >> 3);
    const bool row_ok = i < rb1;
    if (!has_src) {
      if (row_ok)
        for (int e = hl; e < 2 * Rp; e += 8) z[(size_t)2 * i * Rp + e] = src[(size_t)2 * i * Rp + e];
      return;
    }
    int q0 = 0, q1 = 0;
    if (row_ok) {
      q0 = cptr[9 * (size_t)i + sc];
      q1 = cptr[9 * (size_t)i + sc + 1];
    }
    for (int r0 = 0; r0 < Rp; r0 += RB) {
      cx<T> a0[RB], a1[RB];
      for (int q = q0 + hl; q < q1; q += 8) {
        const int cc = __ldg(off_col + q);
        V16 u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = __ldg(Ov + (size_t)q * NV + v);
        const cx<T> *bb = reinterpret_cast<const cx<T> *>(u);
        cx<T> x0[RB], x1[RB];  // colour sc: not written in this step
        ld_rb<T, RB>(z + (size_t)2 * cc * Rp + r0, x0);
        ld_rb<T, RB>(z + ((size_t)2 * cc + 1) * Rp + r0, x1);
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
          a0[rr] = cfma(bb[0], x0[rr], cfma(bb[1], x1[rr], a0[rr]));
          a1[rr] = cfma(bb[2], x0[rr], cfma(bb[3], x1[rr], a1[rr]));
        }
      }
#pragma unroll
      for (int rr = 0; rr < RB; ++rr) {
#pragma unroll
        for (int d = 4; d > 0; d >>= 1) {
          a0[rr] += shfl_down(a0[rr], d);
          a1[rr] += shfl_down(a1[rr], d);
        }
      }
      if (row_ok && hl == 0 && q1 > q0) {
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
          z[(size_t)2 * i * Rp + r0 + rr] -= a0[rr];
          z[((size_t)2 * i + 1) * Rp + r0 + rr] -= a1[rr];
        }
      }
    }
    return;
  }

  // ---- role A: one CTA per box of this colour
  cx<T> *t = reinterpret_cast<cx<T> *>(smem_raw);  // [RB][2n]
  const int b = box0 + blockIdx.x;
  const int s0 = box_start[b], n = box_start[b + 1] - s0;
  cx<T> *t2 = t + (size_t)RB * 2 * n;               // [RB][2n]
  for (int r0 = 0; r0 < Rp; r0 += RB) {
    for (int li = warp; li < n; li += nw) {
      const int i = s0 + li;
      const int q0 = has_src ? cptr[9 * (size_t)i + sc] : 0, q1 = has_src ? cptr[9 * (size_t)i + sc + 1] : 0;
      cx<T> a0[RB], a1[RB];
      for (int q = q0 + lane; q < q1; q += 32) {
        const int cc = __ldg(off_col + q);
        V16 u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = __ldg(Ov + (size_t)q * NV + v);
        const cx<T> *bb = reinterpret_cast<const cx<T> *>(u);
        cx<T> x0[RB], x1[RB];
        ld_rb<T, RB>(z + (size_t)2 * cc * Rp + r0, x0);
        ld_rb<T, RB>(z + ((size_t)2 * cc + 1) * Rp + r0, x1);
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
          a0[rr] = cfma(bb[0], x0[rr], cfma(bb[1], x1[rr], a0[rr]));
          a1[rr] = cfma(bb[2], x0[rr], cfma(bb[3], x1[rr], a1[rr]));
        }
      }
#pragma unroll
      for (int rr = 0; rr < RB; ++rr) {
        const cx<T> u0 = warp_sum(a0[rr]), u1 = warp_sum(a1[rr]);
        if (lane == 0) {
          t[(size_t)rr * 2 * n + 2 * li] = w[(size_t)2 * i * Rp + r0 + rr] - u0;
          t[(size_t)rr * 2 * n + 2 * li + 1] = w[((size_t)2 * i + 1) * Rp + r0 + rr] - u1;
        }
      }
    }
    __syncthreads();
    for (int pass = 0; pass < (both ? 2 : 1); ++pass) {
      const bool lower = forward && pass == 0;
      const cx<T> *M = pass == 0 ? tri + 4 * tri_off[b] : tri2 + 4 * tri2_off[b];
      const cx<T> *in = pass == 0 ? t : t2;
      for (int li = warp; li < n; li += nw) {
        const int j0 = lower ? 0 : li, j1 = lower ? li : n;
        const cx<T> *row = M + 4 * (size_t)(lower ? li * (li - 1) / 2 : li * n - li * (li - 1) / 2);
        cx<T> a0[RB], a1[RB];
        for (int j = j0 + lane; j < j1; j += 32) {
          const cx<T> *B = row + 4 * (j - j0);
          const cx<T> b0 = B[0], b1 = B[1], b2 = B[2], b3 = B[3];
#pragma unroll
          for (int rr = 0; rr < RB; ++rr) {
            const cx<T> x0 = in[(size_t)rr * 2 * n + 2 * j], x1 = in[(size_t)rr * 2 * n + 2 * j + 1];
            a0[rr] = cfma(b0, x0, cfma(b1, x1, a0[rr]));
            a1[rr] = cfma(b2, x0, cfma(b3, x1, a1[rr]));
          }
        }
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
          cx<T> u0 = warp_sum(a0[rr]), u1 = warp_sum(a1[rr]);
          if (lane == 0) {
            if (lower) {
              u0 += in[(size_t)rr * 2 * n + 2 * li];
              u1 += in[(size_t)rr * 2 * n + 2 * li + 1];
            }
            if (both && pass == 0) {
              t2[(size_t)rr * 2 * n + 2 * li] = u0;
              t2[(size_t)rr * 2 * n + 2 * li + 1] = u1;
            } else {
              z[(size_t)2 * (s0 + li) * Rp + r0 + rr] = u0;
              z[((size_t)2 * (s0 + li) + 1) * Rp + r0 + rr] = u1;
            }
          }
        }
      }
      __syncthreads();
    }
  }
}

// [R][m] -> [m][Rp] (zero rows r >= R) and back, in 32 x 32 tiles through shared memory
template <typename T>
__global__ void k_rhs_interleave(int m, int R, int Rp, const cx<T> *__restrict__ a, cx<T> *__restrict__ b) {
  __shared__ __align__(16) unsigned char tile_raw[32 * 33 * sizeof(cx<T>)];  // raw storage: cx has a constructor
  cx<T>(*tile)[33] = reinterpret_cast<cx<T>(*)[33]>(tile_raw);
  const int e0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, e = e0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < R && e < m) ? a[(size_t)r * m + e] : cx<T>();
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int e = e0 + k, r = r0 + threadIdx.x;
    if (e < m && r < Rp) b[(size_t)e * Rp + r] = tile[threadIdx.x][k];
  }
}
template <typename T>
__global__ void k_rhs_deinterleave(int m, int R, int Rp, const cx<T> *__restrict__ b, cx<T> *__restrict__ a) {
  __shared__ __align__(16) unsigned char tile_raw[32 * 33 * sizeof(cx<T>)];  // raw storage: cx has a constructor
  cx<T>(*tile)[33] = reinterpret_cast<cx<T>(*)[33]>(tile_raw);
  const int e0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int e = e0 + k, r = r0 + threadIdx.x;
    tile[k][threadIdx.x] = (e < m && r < Rp) ? b[(size_t)e * Rp + r] : cx<T>();
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, e = e0 + threadIdx.x;
    if (r < R && e < m) a[(size_t)r * m + e] = tile[threadIdx.x][k];
  }
}

// ---------------------------------------------------------------- vectors
__global__ void k_rowscale(int ne, int nrhs, const zd *__restrict__ d, zd *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nrhs * ne * 2) return;
  y[i] = d[i % (2 * (int64_t)ne)] * y[i];
}

__global__ void k_perm_in(int ne, int nrhs, const int *__restrict__ perm, const zd *__restrict__ u, zd *__restrict__ v) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (p >= ne) return;
  int e = perm[p];
  v[((size_t)r * ne + p) * 2] = u[((size_t)r * ne + e) * 2];
  v[((size_t)r * ne + p) * 2 + 1] = u[((size_t)r * ne + e) * 2 + 1];
}
__global__ void k_perm_out(int ne, int nrhs, const int *__restrict__ perm, const zd *__restrict__ v, zd *__restrict__ u) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (p >= ne) return;
  int e = perm[p];
  u[((size_t)r * ne + e) * 2] = v[((size_t)r * ne + p) * 2];
  u[((size_t)r * ne + e) * 2 + 1] = v[((size_t)r * ne + p) * 2 + 1];
}
__global__ void k_d2f(const zd *a, zf *b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = zf((float)a[i].re, (float)a[i].im);
}
__global__ void k_f2d(const zf *a, zd *b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = zd(a[i].re, a[i].im);
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  SIE_REQUIRE(bytes <= 227 * 1024, SIE_EINVAL, "MLFMM interpolation tile exceeds shared memory (too many directions)");
  if (bytes <= 48 * 1024) return;
  // the attribute is raised once per (device, kernel) to the largest size asked for:
  // a driver call per launch costs more host time than some launches take on the GPU
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> raised;
  int dev = 0;
  SIE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  size_t &have = raised[{dev, reinterpret_cast<const void *>(kernel)}];
  if (bytes > have) {
    SIE_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
  }
}

inline int grid1(int64_t n, int bs) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + bs - 1) / bs, 152 * 32)); }

}  // namespace

// ------------------------------------------------------------------ launchers
template <typename T>
void op_near(sie_ctx *c, const cx<T> *x, cx<T> *y, int nrhs, bool accumulate) {
  int warps_per_block = 8;
  int blocks = (c->ne + warps_per_block - 1) / warps_per_block;
  if (nrhs == 1) {
    k_near_spmv<T><<<blocks, 32 * warps_per_block, 0, c->stream>>>(c->ne, nrhs, c->d_row_ptr, c->d_col,
                                                                   (const cx<T> *)tsel<T>::near(c), x, y,
                                                                   accumulate ? 1 : 0);
  } else {
    // right-hand sides per block load: tuned, else 8 (FP32) / 4 (FP64)
    const int rb = c->tune_near_rb ? c->tune_near_rb : (sizeof(T) == 4 ? 8 : 4);
    auto go = [&](auto kern) {
      kern<<<blocks, 32 * warps_per_block, 0, c->stream>>>(c->ne, nrhs, c->d_row_ptr, c->d_col,
                                                          (const cx<T> *)tsel<T>::near(c), x, y, accumulate ? 1 : 0);
    };
    if (rb == 16) go(k_near_spmv_blk<T, 16>);
    else if (rb == 8) go(k_near_spmv_blk<T, 8>);
    else go(k_near_spmv_blk<T, 4>);
  }
  SIE_CHECK_LAUNCH();
  c->launches++;
}

template <typename T, typename TY>
void op_far(sie_ctx *c, const cx<T> *x, cx<TY> *y, int nrhs, bool forked) {
  const int leaf = c->levels - 1;
  const int R = nrhs;
  if (c->levels < 3) return;  // every basis pair is near: no far field
  // The media are independent until the receive: each medium's aggregation,
  // upward pass, translations and downward pass run on a stream of their own
  // (parallel branches when the step is captured as a graph).  For small blocks
  // each branch ends with its medium's receive into the medium's own rows, and
  // a combine adds them into y in medium order; otherwise the receives add into
  // y one medium at a time on the context stream.
  region_streams(c);
  // leaf receive of medium gi on stream rs: into y directly (part = nullptr) or
  // into the medium's rows of d_rpart
  auto receive = [&](size_t gi, cudaStream_t rs, cx<T> *part) {
    RegionHost &G = c->reg[gi];
    LevelHost &LL = G.lev[leaf];
    const size_t per_basis = (size_t)2 * LL.K * sizeof(cx<T>);
    const int cb = (int)std::max<size_t>(1, std::min<size_t>(32, (32 * 1024) / per_basis));  // bases per chunk
    std::complex<double> ie = 1.0 / G.eta;
    // per-row factors of the receive: PMCHWT weights the tangential J-row by
    // eta~ and the M-row by 1/eta~; the other formulations fold theirs into P
    const bool pm = c->form == 3 || c->form == 4;
    const std::complex<double> cj = pm ? G.eta : 1.0, cm = pm ? 1.0 / G.eta : 1.0;
    auto rec = [&](auto kern, int rb) {
      const size_t smem = STAGES * cb * per_basis + (size_t)rb * 4 * LL.K * sizeof(cx<T>);
      set_smem(kern, smem);
      kern<<<LL.nbox, 256, smem, rs>>>(LL.K, c->ne, R, cb, G.d_box_start, G.d_basis_p, (const cx<T> *)tsel<T>::P(G),
                                       (const cx<T> *)LL.d_I, cx<T>((T)G.eta.real(), (T)G.eta.imag()),
                                       cx<T>((T)ie.real(), (T)ie.imag()), y, cx<T>((T)cj.real(), (T)cj.imag()),
                                       cx<T>((T)cm.real(), (T)cm.imag()), part, G.rpart_off, c->rpart_nb);
    };
    // blocks of right-hand sides in the FP32 Krylov operator (not the true
    // residual): split-BF16 products on the tensor cores (sie_set_param key 8)
    const int rec_rb = (std::is_same<T, float>::value && std::is_same<TY, float>::value) ? rec_tc_block(c, R) : 0;
    const bool rec_tc = rec_rb > 0 && !part &&
                        op_receive_tc(c, rec_rb, LL.K, LL.nbox, R, G.d_box_start, G.d_rec_off, G.d_basis_p,
                                      (const unsigned char *)G.d_rec_op, (const zf *)LL.d_I,
                                      zf((float)G.eta.real(), (float)G.eta.imag()),
                                      zf((float)ie.real(), (float)ie.imag()), zf((float)cj.real(), (float)cj.imag()),
                                      zf((float)cm.real(), (float)cm.imag()), (zf *)y, rs);
    if (rec_tc) return;
    // blocks of right-hand sides RB at a time (tuned, else 4) while the box's fields fit in shared memory
    auto fits = [&](int rb) { return STAGES * cb * per_basis + (size_t)rb * 4 * LL.K * sizeof(cx<T>) <= 227 * 1024; };
    int rb = R == 1 ? 1 : (c->tune_rec_rb ? c->tune_rec_rb : 4);
    while (rb > 1 && !fits(rb)) rb /= 2;
    if (rb == 4) rec(k_disaggregate<T, 4, TY>, 4);
    else if (rb == 2) rec(k_disaggregate<T, 2, TY>, 2);
    else rec(k_disaggregate<T, 1, TY>, 1);
    SIE_CHECK_LAUNCH();
    c->launches++;
  };
  // small blocks in the SIMT receive: the media's receives run concurrently,
  // each in its own branch, and a combine adds them into y in medium order
  const int rec_rb0 = (std::is_same<T, float>::value && std::is_same<TY, float>::value) ? rec_tc_block(c, R) : 0;
  const bool par = rec_rb0 == 0 && R <= c->rpart_cap && c->d_rpart != nullptr && c->d_rmap != nullptr;
  if (!forked) SIE_CUDA(cudaEventRecord(c->ev_fork, c->stream));
  for (size_t gi = 0; gi < c->reg.size(); ++gi) {
    RegionHost &G = c->reg[gi];
    if (G.nb == 0) continue;
    cudaStream_t st = c->rstream[gi];
    SIE_CUDA(cudaStreamWaitEvent(st, c->ev_fork, 0));
    LevelHost &LL = G.lev[leaf];
    // aggregation at the leaf level
    const size_t per_basis = (size_t)2 * LL.K * sizeof(cx<T>);
    const int cb = (int)std::max<size_t>(1, std::min<size_t>(32, (32 * 1024) / per_basis));  // bases per chunk
    SIE_REQUIRE(LL.K <= 4 * 256, SIE_EINVAL, "MLFMM: too many leaf directions for the aggregation kernel");
    {
      auto agg = [&](auto kern, int rb) {
        const size_t smem = STAGES * cb * per_basis + (size_t)G.max_leaf * rb * 2 * sizeof(cx<T>);
        set_smem(kern, smem);
        kern<<<LL.nbox, 256, smem, st>>>(LL.K, c->ne, R, cb, G.d_box_start, G.d_basis_p, G.d_basis_sign,
                                                (const cx<T> *)tsel<T>::V(G), x, (cx<T> *)LL.d_S);
      };
      // blocks of right-hand sides in the FP32 operator: split-BF16 products on
      // the tensor cores (not in the true-residual operator, TY = double, whose
      // accuracy floor decides convergence: there the FP32 SIMT kernel)
      const int tc_rb = (std::is_same<T, float>::value && std::is_same<TY, float>::value) ? agg_tc_block(c, R) : 0;
      const bool tc = tc_rb > 0 && op_aggregate_tc(c, tc_rb, LL.K, LL.nbox, G.max_leaf, R, G.d_box_start,
                                                   G.d_agg_off, G.d_basis_p, G.d_basis_sign,
                                                   (const unsigned char *)G.d_agg_op, (const zf *)x, (zf *)LL.d_S, st);
      if (!tc) {
        // more than 512 leaf directions: four per thread, one right-hand side per pass
        if (LL.K > 2 * 256) agg(k_aggregate<T, 1, 4>, 1);
        else if (R == 1) agg(k_aggregate<T, 1, 2>, 1);
        else agg(k_aggregate<T, 4, 2>, 4);
        SIE_CHECK_LAUNCH();
        c->launches++;
      }
    }
    // upward pass: interpolate + shift each child, then sum into parents
    for (int lv = leaf; lv > G.top; --lv) {
      LevelHost &C = G.lev[lv], &P = G.lev[lv - 1];
      const int nthc = C.L + 1, Nc = 2 * C.L + 2, Np = 2 * P.L + 2, nthp = P.L + 1;
      const size_t tabs = ((size_t)Np * Nc + 2 * (size_t)nthp * nthc) * sizeof(T);
      // one source (J or M) per pass: fewer registers, more CTAs per SM (measured
      // faster than both at once); the parent's column pairs in chunks of cw
      // (all of them when they fit in shared memory; the tables read from
      // global memory when even one column pair does not fit beside them)
      auto smem_for = [&](int cw, bool gt) {
        return ((size_t)3 * C.K + (size_t)3 * nthc * 2 * cw) * sizeof(cx<T>) + (gt ? 0 : tabs);
      };
      int cw = P.L + 1;
      bool gt = false;
      while (cw > 1 && smem_for(cw, false) > 200 * 1024) cw = (cw + 1) / 2;
      if (smem_for(cw, false) > 227 * 1024) {
        gt = true;
        cw = P.L + 1;
        while (cw > 1 && smem_for(cw, true) > 200 * 1024) cw = (cw + 1) / 2;
      }
      const size_t smem = smem_for(cw, gt);
      cx<T> *Y = (cx<T> *)((char *)c->d_scratch + gi * c->scratch_region);
      // the sources J, M as a grid dimension for one right-hand side on the
      // smaller levels: more CTAs in flight and a shorter chain per CTA
      // (measured: far field 0.522 -> 0.515 ms on the coated sphere, 0.163 ->
      // 0.153 ms on the nanoparticle; slower from 4 right-hand sides on)
      const int zsplit = c->tune_interp_split >= 0 ? c->tune_interp_split : (R == 1 && C.nbox < 2048 ? 1 : 0);
      dim3 grid(C.nbox, R, zsplit ? 2 : 1);
      // threads sized to the larger task list (phi step: theta rows x column pairs;
      // theta step: row pairs x column pairs), so small levels fit more CTAs per SM
      const int tasks = std::max(nthc * cw, (nthp + 1) / 2 * cw);
      const int threads = std::min(256, std::max(64, (tasks + 31) / 32 * 32));
      if (cw == P.L + 1 && !gt) {  // the whole parent sampling at once: the single-pass kernel
        set_smem(k_interp_up<T, 1>, smem);
        k_interp_up<T, 1><<<grid, threads, smem, st>>>(
            C.K, C.L, P.K, P.L, R, C.d_oct, (const T *)tsel<T>::tp(C), (const T *)tsel<T>::tp(P),
            (const T *)tsel<T>::Phi(P), (const T *)tsel<T>::Thp(P), (const T *)tsel<T>::Thm(P),
            (const cx<T> *)tsel<T>::up(P), (const cx<T> *)C.d_S, Y);
      } else {
        auto kern = gt ? k_interp_up_chunked<T, 1, true> : k_interp_up_chunked<T, 1, false>;
        set_smem(kern, smem);
        kern<<<grid, threads, smem, st>>>(
            C.K, C.L, P.K, P.L, R, cw, C.d_oct, (const T *)tsel<T>::tp(C), (const T *)tsel<T>::tp(P),
            (const T *)tsel<T>::Phi(P), (const T *)tsel<T>::Thp(P), (const T *)tsel<T>::Thm(P),
            (const cx<T> *)tsel<T>::up(P), (const cx<T> *)C.d_S, Y);
      }
      SIE_CHECK_LAUNCH();
      k_up_sum<T><<<dim3((P.K + 127) / 128, P.nbox), 128, 0, st>>>(P.K, R, P.d_ch_ptr, P.d_ch_idx, Y,
                                                                           (cx<T> *)P.d_S);
      SIE_CHECK_LAUNCH();
      c->launches += 2;
    }
    // translations at every level: per target box for few right-hand sides (more
    // CTAs in flight), by sibling groups for blocks of 8 or more (fewer loads)
    for (int lv = G.top; lv <= leaf; ++lv) {
      LevelHost &B = G.lev[lv];
      const bool by_group = B.ngroups > 0 && (c->tune_m2l >= 0 ? (c->tune_m2l == 1 && R >= 2) : R >= 8);
      // (split groups measured slower than per target box for one right-hand side: 0.603 vs 0.558 ms far field)
      const bool by_split = B.ngroups > 0 && !by_group && c->tune_m2l == 2;
      if (by_split) {
        // sibling groups split over 4 warps, 32 directions per CTA
        SIE_REQUIRE(B.ngroups <= 65535 && R <= 65535, SIE_EINVAL, "MLFMM: too many sibling groups for one launch");
        constexpr int SW = 4;
        const size_t smem = (size_t)(SW - 1) * 8 * 4 * 32 * sizeof(cx<T>) + (size_t)B.max_group_entries * 10 * sizeof(int);
        set_smem(k_m2l_split<T, SW>, smem);
        k_m2l_split<T, SW><<<dim3((B.K + 31) / 32, B.ngroups, R), 32 * SW, smem, st>>>(
            B.K, R, B.d_grp_ptr, B.d_grp_box, B.d_grp_ent, (const cx<T> *)tsel<T>::Tr(B), (const cx<T> *)B.d_S,
            (cx<T> *)B.d_I);
      } else if (by_group) {
        SIE_REQUIRE(B.ngroups <= 65535 && R <= 65535, SIE_EINVAL, "MLFMM: too many sibling groups for one launch");
        dim3 grid((B.K + 127) / 128, B.ngroups, R);
        const size_t smem = (size_t)B.max_group_entries * 10 * sizeof(int);
        set_smem(k_m2l_group<T>, smem);
        k_m2l_group<T><<<grid, 128, smem, st>>>(B.K, R, B.d_grp_ptr, B.d_grp_box, B.d_grp_ent,
                                                       (const cx<T> *)tsel<T>::Tr(B), (const cx<T> *)B.d_S,
                                                       (cx<T> *)B.d_I);
      } else {
        SIE_REQUIRE((B.K + 31) / 32 <= 65535, SIE_EINVAL, "MLFMM: too many directions for one launch");
        dim3 grid(B.nbox, (B.K + 31) / 32);
        k_m2l<T><<<grid, 32, 0, st>>>(B.nbox, B.K, R, B.d_il_ptr, B.d_il_src, B.d_il_slot,
                                              (const cx<T> *)tsel<T>::Tr(B), (const cx<T> *)B.d_S, (cx<T> *)B.d_I);
      }
      SIE_CHECK_LAUNCH();
      c->launches++;
    }
    // downward pass: shift + anterpolate (exact transpose) into children
    for (int lv = G.top; lv < leaf; ++lv) {
      LevelHost &P = G.lev[lv], &C = G.lev[lv + 1];
      const int nthc = C.L + 1, Nc = 2 * C.L + 2, Np = 2 * P.L + 2, nthp = P.L + 1;
      const size_t tabs = ((size_t)Np * Nc + 2 * (size_t)nthp * nthc) * sizeof(T);
      // one source (J or M) per pass; the parent's column pairs in chunks of cw
      // (all of them when they fit in shared memory)
      auto smem_for = [&](int cw, bool gt) {
        return ((size_t)3 * nthp * 2 * cw + (size_t)3 * nthc * 2 * cw) * sizeof(cx<T>) + (gt ? 0 : tabs);
      };
      int cw = P.L + 1;
      bool gt = false;
      while (cw > 1 && smem_for(cw, false) > 200 * 1024) cw = (cw + 1) / 2;
      if (smem_for(cw, false) > 227 * 1024) {
        gt = true;
        cw = P.L + 1;
        while (cw > 1 && smem_for(cw, true) > 200 * 1024) cw = (cw + 1) / 2;
      }
      const size_t smem = smem_for(cw, gt);
      const int zsplit = c->tune_interp_split >= 0 ? c->tune_interp_split : (R == 1 && C.nbox < 2048 ? 1 : 0);
      dim3 grid(C.nbox, R, zsplit ? 2 : 1);
      const int tasks = std::max((nthc + 1) / 2 * cw, nthc * (C.L + 1));
      const int threads = std::min(256, std::max(64, (tasks + 31) / 32 * 32));
      if (cw == P.L + 1 && !gt) {  // the whole parent sampling at once: the single-pass kernel
        set_smem(k_anterp_dn<T, 1>, smem);
        k_anterp_dn<T, 1><<<grid, threads, smem, st>>>(
            C.K, C.L, P.K, P.L, R, C.d_parent, C.d_oct, (const T *)tsel<T>::tp(C), (const T *)tsel<T>::tp(P),
            (const T *)tsel<T>::Phi(P), (const T *)tsel<T>::Thp(P), (const T *)tsel<T>::Thm(P),
            (const cx<T> *)tsel<T>::dn(P), (const cx<T> *)P.d_I, (cx<T> *)C.d_I);
      } else {
        auto kern = gt ? k_anterp_dn_chunked<T, 1, true> : k_anterp_dn_chunked<T, 1, false>;
        set_smem(kern, smem);
        kern<<<grid, threads, smem, st>>>(
            C.K, C.L, P.K, P.L, R, cw, C.d_parent, C.d_oct, (const T *)tsel<T>::tp(C), (const T *)tsel<T>::tp(P),
            (const T *)tsel<T>::Phi(P), (const T *)tsel<T>::Thp(P), (const T *)tsel<T>::Thm(P),
            (const cx<T> *)tsel<T>::dn(P), (const cx<T> *)P.d_I, (cx<T> *)C.d_I);
      }
      SIE_CHECK_LAUNCH();
      c->launches++;
    }
    if (par) receive(gi, st, (cx<T> *)c->d_rpart);
    SIE_CUDA(cudaEventRecord(c->ev_join[gi], st));
  }
  if (par) {
    // every medium's rows are in d_rpart: add them into y in medium order
    for (size_t gi = 0; gi < c->reg.size(); ++gi)
      if (c->reg[gi].nb > 0) SIE_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join[gi], 0));
    const int64_t n = (int64_t)R * c->ne;
    k_rec_combine<T, TY><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->ne, R, c->rpart_nb, c->d_rmap,
                                                                            (const cx<T> *)c->d_rpart, y);
    SIE_CHECK_LAUNCH();
    c->launches++;
    return;
  }
  for (size_t gi = 0; gi < c->reg.size(); ++gi) {
    RegionHost &G = c->reg[gi];
    if (G.nb == 0) continue;
    SIE_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join[gi], 0));
    receive(gi, c->stream, nullptr);
  }
}

template <typename T>
void op_ilu(sie_ctx *c, const cx<T> *r, cx<T> *z, int nrhs) {
  IluHost &I = c->ilu;
  const int mb = std::max(I.max_box, 1);
  if (nrhs == 1) {
    constexpr int NT = 512, NW = NT / 32;
    const size_t base = ((size_t)NW * 2 * mb + 4 * (size_t)mb) * sizeof(cx<T>) + (2 * (size_t)mb + 1) * sizeof(int) + 16;
    const size_t trib = (size_t)mb * (mb + 1) / 2 * 4 * sizeof(cx<T>);
    const int stage = base + trib <= 100 * 1024 ? 1 : 0;
    const size_t smem = base + (stage ? trib : 0);
    auto rows_from = [&](int colr) { return c->leaf_start[I.colour_ptr[colr]]; };
    if (c->ilu_schedule == 0) {
      // the 15 steps in one cooperative launch of as many CTAs as fit on the GPU at once
      auto kern = k_ilu_persistent<T, NT>;
      set_smem(kern, smem);
      static std::mutex mu;
      static std::map<std::pair<int, size_t>, int> grid_of;  // (device, shared bytes) -> resident CTAs
      int dev = 0;
      SIE_CUDA(cudaGetDevice(&dev));
      int grid = 0;
      {
        std::lock_guard<std::mutex> lock(mu);
        int &g = grid_of[{dev * 2 + (sizeof(T) == 4 ? 1 : 0), smem}];
        if (g == 0) {
          int per_sm = 0, nsm = 0;
          SIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
          SIE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
          SIE_REQUIRE(per_sm >= 1, SIE_EINVAL, "ILU(0) apply: the sweep kernel does not fit on one SM");
          g = per_sm * nsm;
        }
        grid = g;
      }
      IluPlan P = {};
      P.nsteps = 0;
      for (int step = 0; step < 15; ++step) {
        const bool fwd = step < 8;
        const int colr = fwd ? step : 14 - step;
        const int np = I.piece_ptr[step + 1] - I.piece_ptr[step];
        const int rb0 = fwd ? rows_from(colr + 1) : 0, rb1 = fwd ? c->ne : rows_from(colr);
        const int nitems = np + (rb1 - rb0 + (32 / ILU_RL) * NW - 1) / ((32 / ILU_RL) * NW);
        if (nitems == 0) continue;
        IluStepDesc &D = P.s[P.nsteps++];
        D.forward = fwd ? 1 : 0;
        D.both = colr == 7 ? 1 : 0;
        D.colour = colr;
        D.npieceA = np;
        D.piece0 = I.piece_ptr[step];
        D.rb0 = rb0;
        D.rb1 = rb1;
        D.nitems = nitems;
        D.cptr = fwd ? I.d_lo_cptr : I.d_up_cptr;
        D.col = fwd ? I.d_lo_col : I.d_up_col;
        D.val = fwd ? tsel<T>::lo(I) : tsel<T>::upv(I);
        D.tri_off = fwd ? I.d_tl_off : I.d_tu_off;
        D.tri = fwd ? tsel<T>::tl(I) : tsel<T>::tu(I);
      }
      SIE_CUDA(cudaMemsetAsync(I.d_bar, 0, sizeof(unsigned), c->stream));
      SIE_CUDA(launch_cooperative(kern, dim3(grid), dim3(NT), smem, c->stream, P, (const int *)I.d_pieces, stage, mb,
                                  (cx<T> *)I.d_piece_scratch, I.d_piece_count, (const int *)I.d_box_start,
                                  (const int64_t *)I.d_tu_off, (const cx<T> *)tsel<T>::tu(I), (const cx<T> *)r, z,
                                  I.d_bar, c->wait_limit, c->d_err));
      SIE_CHECK_LAUNCH();
      c->launches++;
      return;
    }
    set_smem(k_ilu_sweep<T, NT>, smem);
    // forward colours 0..7 (the last also applies U^{-1}), then backward 6..0
    for (int step = 0; step < 15; ++step) {
      const bool fwd = step < 8;
      const int colr = fwd ? step : 14 - step;
      const int np = I.piece_ptr[step + 1] - I.piece_ptr[step];
      const int rb0 = fwd ? rows_from(colr + 1) : 0, rb1 = fwd ? c->ne : rows_from(colr);
      const int nrowB = rb1 - rb0;
      const int grid = np + (nrowB + (32 / ILU_RL) * NW - 1) / ((32 / ILU_RL) * NW);
      if (grid == 0) continue;
      // each step may launch while the previous one drains (programmatic
      // dependent launch; the kernel waits before it reads z)
      SIE_CUDA(launch_chained(
          ILU_PDL, k_ilu_sweep<T, NT>, dim3(grid), dim3(NT), smem, c->stream, fwd ? 1 : 0, colr == 7 ? 1 : 0, colr, np,
          (const int *)(I.d_pieces + 5 * (size_t)I.piece_ptr[step]), rb0, rb1, stage, mb,
          (cx<T> *)I.d_piece_scratch, I.d_piece_count, (const int *)I.d_box_start,
          (const int *)(fwd ? I.d_lo_cptr : I.d_up_cptr), (const int *)(fwd ? I.d_lo_col : I.d_up_col),
          (const cx<T> *)(fwd ? tsel<T>::lo(I) : tsel<T>::upv(I)), (const int64_t *)(fwd ? I.d_tl_off : I.d_tu_off),
          (const cx<T> *)(fwd ? tsel<T>::tl(I) : tsel<T>::tu(I)), (const int64_t *)I.d_tu_off,
          (const cx<T> *)tsel<T>::tu(I), (const cx<T> *)r, z));
      SIE_CHECK_LAUNCH();
      c->launches++;
    }
    return;
  }
  // block of right-hand sides: the same 15 steps, RB right-hand sides per block
  // load (tuned, else 8 in FP32 and 4 in FP64)
  const int rbq = c->tune_ilu_rb ? c->tune_ilu_rb : (sizeof(T) == 4 ? 8 : 4);
  auto sweeps = [&](auto kern, int RB) {
    const size_t smem = 2 * (size_t)RB * 2 * mb * sizeof(cx<T>);
    set_smem(kern, smem);
    auto rows_from = [&](int colr) { return c->leaf_start[I.colour_ptr[colr]]; };
    for (int step = 0; step < 15; ++step) {
      const bool fwd = step < 8;
      const int colr = fwd ? step : 14 - step;
      const int first = I.colour_ptr[colr], cnt = I.colour_ptr[colr + 1] - first;
      const int rb0 = fwd ? rows_from(colr + 1) : 0, rb1 = fwd ? c->ne : rows_from(colr);
      const int grid = cnt + (rb1 - rb0 + 31) / 32;  // role B: 32 rows per 256-thread CTA
      if (grid == 0) continue;
      kern<<<grid, 256, smem, c->stream>>>(
          c->ne, nrhs, fwd ? 1 : 0, colr == 7 ? 1 : 0, colr, cnt, first, rb0, rb1, I.d_box_start,
          fwd ? I.d_lo_cptr : I.d_up_cptr, fwd ? I.d_lo_col : I.d_up_col,
          (const cx<T> *)(fwd ? tsel<T>::lo(I) : tsel<T>::upv(I)), fwd ? I.d_tl_off : I.d_tu_off,
          (const cx<T> *)(fwd ? tsel<T>::tl(I) : tsel<T>::tu(I)), I.d_tu_off, (const cx<T> *)tsel<T>::tu(I), r, z);
      SIE_CHECK_LAUNCH();
      c->launches++;
    }
  };
  const int RBu = (rbq == 16 && 2 * (size_t)16 * 2 * mb * sizeof(cx<T>) <= 227 * 1024) ? 16 : rbq >= 8 ? 8 : 4;
  // with the context's work buffers: the sweeps on right-hand-side-interleaved
  // copies of r and z (contiguous gathers); without them (the allocation-free
  // entry on a context that never ran a block) on r and z as they are
  const int Rp = (nrhs + RBu - 1) / RBu * RBu, m = 2 * c->ne;
  if (c->d_iluT && Rp <= c->iluT_R) {
    cx<T> *rT = (cx<T> *)c->d_iluT, *zT = rT + (size_t)Rp * m;
    const dim3 tg((m + 31) / 32, (Rp + 31) / 32), tb(32, 8);
    k_rhs_interleave<T><<<tg, tb, 0, c->stream>>>(m, nrhs, Rp, r, rT);
    SIE_CHECK_LAUNCH();
    auto sweepsT = [&](auto kern) {
      const size_t smem = 2 * (size_t)RBu * 2 * mb * sizeof(cx<T>);
      set_smem(kern, smem);
      auto rows_from = [&](int colr) { return c->leaf_start[I.colour_ptr[colr]]; };
      for (int step = 0; step < 15; ++step) {
        const bool fwd = step < 8;
        const int colr = fwd ? step : 14 - step;
        const int first = I.colour_ptr[colr], cnt = I.colour_ptr[colr + 1] - first;
        const int rb0 = fwd ? rows_from(colr + 1) : 0, rb1 = fwd ? c->ne : rows_from(colr);
        const int grid = cnt + (rb1 - rb0 + 31) / 32;  // role B: 32 rows per 256-thread CTA
        if (grid == 0) continue;
        kern<<<grid, 256, smem, c->stream>>>(
            c->ne, Rp, fwd ? 1 : 0, colr == 7 ? 1 : 0, colr, cnt, first, rb0, rb1, I.d_box_start,
            fwd ? I.d_lo_cptr : I.d_up_cptr, fwd ? I.d_lo_col : I.d_up_col,
            (const cx<T> *)(fwd ? tsel<T>::lo(I) : tsel<T>::upv(I)), fwd ? I.d_tl_off : I.d_tu_off,
            (const cx<T> *)(fwd ? tsel<T>::tl(I) : tsel<T>::tu(I)), I.d_tu_off, (const cx<T> *)tsel<T>::tu(I),
            (const cx<T> *)rT, zT);
        SIE_CHECK_LAUNCH();
        c->launches++;
      }
    };
    if (RBu == 16) sweepsT(k_ilu_sweep_blkT<T, 16>);
    else if (RBu == 8) sweepsT(k_ilu_sweep_blkT<T, 8>);
    else sweepsT(k_ilu_sweep_blkT<T, 4>);
    k_rhs_deinterleave<T><<<tg, tb, 0, c->stream>>>(m, nrhs, Rp, zT, z);
    SIE_CHECK_LAUNCH();
    c->launches += 2;
    return;
  }
  if (RBu == 16) sweeps(k_ilu_sweep_blk<T, 16>, 16);
  else if (RBu == 8) sweeps(k_ilu_sweep_blk<T, 8>, 8);
  else sweeps(k_ilu_sweep_blk<T, 4>, 4);
}

void op_permute_in(sie_ctx *c, const zd *u, zd *v, int nrhs) {
  dim3 grid((c->ne + 255) / 256, nrhs);
  k_perm_in<<<grid, 256, 0, c->stream>>>(c->ne, nrhs, c->d_perm, u, v);
  SIE_CHECK_LAUNCH();
  c->launches++;
}
void op_permute_out(sie_ctx *c, const zd *v, zd *u, int nrhs) {
  dim3 grid((c->ne + 255) / 256, nrhs);
  k_perm_out<<<grid, 256, 0, c->stream>>>(c->ne, nrhs, c->d_perm, v, u);
  SIE_CHECK_LAUNCH();
  c->launches++;
}
void op_d2f(sie_ctx *c, const zd *a, zf *b, int64_t n) {
  k_d2f<<<grid1(n, 256), 256, 0, c->stream>>>(a, b, n);
  SIE_CHECK_LAUNCH();
  c->launches++;
}
void op_f2d(sie_ctx *c, const zf *a, zd *b, int64_t n) {
  k_f2d<<<grid1(n, 256), 256, 0, c->stream>>>(a, b, n);
  SIE_CHECK_LAUNCH();
  c->launches++;
}

// marks on the context stream where the media's far-field passes may start
void far_fork(sie_ctx *c) {
  region_streams(c);
  SIE_CUDA(cudaEventRecord(c->ev_fork, c->stream));
}

void op_rowscale(sie_ctx *c, zd *y, int nrhs) {
  if (c->form != 4 || !c->d_rowscale) return;
  const int64_t n = (int64_t)nrhs * c->ne * 2;
  k_rowscale<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->ne, nrhs, (const zd *)c->d_rowscale, y);
  SIE_CHECK_LAUNCH();
  c->launches++;
}

void apply_matvec(sie_ctx *c, const zd *x, zd *y, int nrhs, sie_prec prec, int parts) {
  int64_t n = (int64_t)nrhs * c->ne * 2;
  if (prec == SIE_PREC_FP64) {
    // the media's far-field passes start first and overlap the near-field product
    if (parts & 2) far_fork(c);
    if (parts & 1) op_near<double>(c, x, y, nrhs, false);
    else SIE_CUDA(cudaMemsetAsync(y, 0, n * sizeof(zd), c->stream));
    if (parts & 2) op_far<double>(c, x, y, nrhs, true);
  } else if (prec == SIE_PREC_NEAR64) {
    // FP64 near field; the far field from an FP32 copy of x, its receives
    // adding into the FP64 product
    zf *xf = (zf *)c->d_xf;
    if (parts & 2) op_d2f(c, x, xf, n);
    if (parts & 2) far_fork(c);
    if (parts & 1) op_near<double>(c, x, y, nrhs, false);
    else SIE_CUDA(cudaMemsetAsync(y, 0, n * sizeof(zd), c->stream));
    if (parts & 2) op_far<float, double>(c, xf, y, nrhs, true);
  } else {
    zf *xf = (zf *)c->d_xf, *yf = (zf *)c->d_yf;
    op_d2f(c, x, xf, n);
    if (parts & 2) far_fork(c);
    if (parts & 1) op_near<float>(c, xf, yf, nrhs, false);
    else SIE_CUDA(cudaMemsetAsync(yf, 0, n * sizeof(zf), c->stream));
    if (parts & 2) op_far<float>(c, xf, yf, nrhs, true);
    op_f2d(c, yf, y, n);
  }
  op_rowscale(c, y, nrhs);  // ICTF: D (N + F) x
}

void apply_ilu(sie_ctx *c, const zd *r, zd *z, int nrhs, sie_prec prec) {
  int64_t n = (int64_t)nrhs * c->ne * 2;
  if (prec == SIE_PREC_FP64) {
    op_ilu<double>(c, r, z, nrhs);
  } else {
    zf *rf = (zf *)c->d_xf, *zf_ = (zf *)c->d_yf;
    op_d2f(c, r, rf, n);
    op_ilu<float>(c, rf, zf_, nrhs);
    op_f2d(c, zf_, z, n);
  }
}

template void op_near<double>(sie_ctx *, const zd *, zd *, int, bool);
template void op_near<float>(sie_ctx *, const zf *, zf *, int, bool);
template void op_far<double, double>(sie_ctx *, const zd *, zd *, int, bool);
template void op_far<float, float>(sie_ctx *, const zf *, zf *, int, bool);
template void op_far<float, double>(sie_ctx *, const zf *, zd *, int, bool);
template void op_ilu<double>(sie_ctx *, const zd *, zd *, int);
template void op_ilu<float>(sie_ctx *, const zf *, zf *, int);
