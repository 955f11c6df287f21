// Learned right preconditioner: one MLP 128 -> 256 -> 256 -> 128 (ReLU) shared
// by all leaf chunks (<= 32 bases of one leaf box, 64 complex unknowns).
// Applied after ILU(0) inside flexible GMRES, u = ILU^-1 v:
//     z_c = u_c + |u_c| NN(u_c / |u_c|)
// trained on residual/error pairs (r_k, e_k = x* - x_k) that the solver
// records at its restarts, with input u = ILU^-1 r_k and target
// (e_k - u)_c / |u_c|: a learned local correction of the ILU output.  Weights and
// activations are stored in BF16, products accumulate in FP32, Adam keeps FP32
// master weights.  Every step runs in the kernels below.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>

#include <type_traits>

#include "common.h"

namespace {

typedef __nv_bfloat16 bf16;
constexpr int D0 = 128, D1 = 256, D2 = 256, D3 = 128;
constexpr int CH = 32;  // bases per chunk

__device__ __forceinline__ float ld(const float *p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld(const bf16 *p, size_t i) { return __bfloat162float(p[i]); }

// ---------------------------------------------------------------- chunks
// X[s][128] = (re, im of the chunk's unknowns) / |v_c|, zero padded; nrm[s] = |v_c|.
__global__ void k_chunk_gather(int nchunk, const int *__restrict__ cstart, const int *__restrict__ clen,
                               const zd *__restrict__ v, bf16 *__restrict__ X, float *__restrict__ nrm) {
  int c = blockIdx.x;
  int t = threadIdx.x;  // 128 threads: one real component each
  __shared__ float red[128];
  int s0 = cstart[c], n = clen[c];
  float val = 0.f;
  if (t < 4 * n) {
    zd z = v[2 * (size_t)s0 + (t >> 1)];
    val = (float)((t & 1) ? z.im : z.re);
  }
  red[t] = val * val;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  float nn = sqrtf(red[0]);
  float inv = nn > 0.f ? 1.f / nn : 0.f;
  X[(size_t)c * D0 + t] = __float2bfloat16(val * inv);
  if (t == 0) nrm[c] = nn;
}

// target T[s] = (e - z_ilu) restricted to the chunk / |r_c|
__global__ void k_chunk_target(int nchunk, const int *__restrict__ cstart, const int *__restrict__ clen,
                               const zd *__restrict__ e, const zd *__restrict__ z, const float *__restrict__ nrm,
                               float *__restrict__ Tt) {
  int c = blockIdx.x, t = threadIdx.x;
  int s0 = cstart[c], n = clen[c];
  float val = 0.f;
  if (t < 4 * n && nrm[c] > 0.f) {
    size_t i = 2 * (size_t)s0 + (t >> 1);
    double d = (t & 1) ? e[i].im - z[i].im : e[i].re - z[i].re;
    val = (float)(d / nrm[c]);
  }
  Tt[(size_t)c * D3 + t] = val;
}

// z_c += |v_c| * Y_c
__global__ void k_chunk_scatter(int nchunk, const int *__restrict__ cstart, const int *__restrict__ clen,
                                const float *__restrict__ Y, const float *__restrict__ nrm, zd *__restrict__ z) {
  int c = blockIdx.x, t = threadIdx.x;
  int s0 = cstart[c], n = clen[c];
  if (t < 2 * n) {
    size_t i = 2 * (size_t)s0 + t;
    float a = nrm[c];
    z[i].re += (double)(a * Y[(size_t)c * D3 + 2 * t]);
    z[i].im += (double)(a * Y[(size_t)c * D3 + 2 * t + 1]);
  }
}

// ---------------------------------------------------------------- dense layers
// C[M][N] = act(sum_k A(i,k) B(k,j) + bias[j]) with FP32 accumulation.
// A(i,k) = A[ta ? k*lda + i : i*lda + k], B(k,j) = B[tb ? j*ldb + k : k*ldb + j].
// Writes C as FP32 (Cf) and/or BF16 (Cb); relu != 0 applies max(0, .).
// Split over K (gridDim.z > 1, kch inner indices per slice): slice z adds
// k in [z kch, min(K, (z + 1) kch)) and writes its raw partial tile to
// Cf + z M N (no bias or activation); k_splitk_sum adds the slices in order.
template <typename TA, typename TB>
__global__ void k_dense(int M, int N, int K, int kch, const TA *__restrict__ A, int lda, int ta,
                        const TB *__restrict__ B, int ldb, int tb, const float *__restrict__ bias, int relu,
                        float *__restrict__ Cf, bf16 *__restrict__ Cb) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kb = blockIdx.z * kch, ke = min(K, kb + kch);
  if (gridDim.z > 1) {
    Cf += (size_t)blockIdx.z * M * N;
    bias = nullptr;
    relu = 0;
    Cb = nullptr;
  }
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      int kk, mm;
      if (ta) { mm = t % 64; kk = t / 64; } else { kk = t % 16; mm = t / 16; }
      int gi = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gi < M && gk < ke) ? ld(A, ta ? (size_t)gk * lda + gi : (size_t)gi * lda + gk) : 0.f;
    }
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      int kk, nn;
      if (tb) { kk = t % 16; nn = t / 16; } else { nn = t % 64; kk = t / 64; }
      int gj = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gj < N && gk < ke) ? ld(B, tb ? (size_t)gj * ldb + gk : (size_t)gk * ldb + gj) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < M && gj < N) {
        float v = acc[i][j] + (bias ? bias[gj] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        if (Cf) Cf[(size_t)gi * N + gj] = v;
        if (Cb) Cb[(size_t)gi * N + gj] = __float2bfloat16(v);
      }
    }
}

// C = act(sum_z P[z] + bias), the slices of a split-K product added in order
__global__ void k_splitk_sum(int64_t mn, int N, int S, const float *__restrict__ P, const float *__restrict__ bias,
                             int relu, float *__restrict__ Cf, bf16 *__restrict__ Cb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mn) return;
  float v = 0.f;
  for (int z = 0; z < S; ++z) v += P[(size_t)z * mn + i];
  if (bias) v += bias[i % N];
  if (relu) v = fmaxf(v, 0.f);
  if (Cf) Cf[i] = v;
  if (Cb) Cb[i] = __float2bfloat16(v);
}

// dH = dY .* (H > 0) in place (H stored in BF16)
__global__ void k_relu_mask(int64_t n, const bf16 *__restrict__ H, float *__restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(__bfloat162float(H[i]) > 0.f)) d[i] = 0.f;
}

// dY = w (Y - T) / n and per-block partial losses sum w (Y - T)^2 / (2n);
// w = per-sample weight (null: 1)
__global__ void k_mse(int64_t n_el, float inv_n, const float *__restrict__ Y, const float *__restrict__ T,
                      const float *__restrict__ wt, float *__restrict__ dY, double *__restrict__ loss) {
  __shared__ double red[256];
  double acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += (int64_t)gridDim.x * blockDim.x) {
    float d = Y[i] - T[i];
    float w = wt ? wt[i / D3] : 1.f;
    dY[i] = w * d * inv_n;
    acc += 0.5 * (double)w * d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv_n);
}

// db[j] = sum_i dY[i][j]
__global__ void k_colsum(int M, int N, const float *__restrict__ dY, float *__restrict__ db) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float acc = 0.f;
  for (int i = 0; i < M; ++i) acc += dY[(size_t)i * N + j];
  db[j] = acc;
}

// Adam on FP32 master parameters; refreshes the BF16 weight copy.
__global__ void k_adam(int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       const float *__restrict__ g, float *__restrict__ w, float *__restrict__ m,
                       float *__restrict__ v, bf16 *__restrict__ wb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}

// weighted dots[0] += <Y,T>, dots[1] += <Y,Y>, dots[2] += <T,T>
__global__ void k_dots(int64_t n, const float *__restrict__ Y, const float *__restrict__ T,
                       const float *__restrict__ wt, double *dots) {
  __shared__ double red[3][256];
  double a = 0, b = 0, cc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double y = Y[i], t = T[i], w = wt[i / D3];
    a += w * y * t;
    b += w * y * y;
    cc += w * t * t;
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = cc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) atomicAdd(dots + q, red[q][0]);
}

// sample weights of one pair: |u_c|^2 normalised to mean 1 over the pair's chunks,
// so that the loss measures the error of the corrected z itself
__global__ void k_pair_weights(int nchunk, const float *__restrict__ nrm, float *__restrict__ wt) {
  __shared__ double red[256];
  const float *a = nrm + (size_t)blockIdx.x * nchunk;
  float *w = wt + (size_t)blockIdx.x * nchunk;
  double acc = 0;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) acc += (double)a[c] * a[c];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double tot = red[0];
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x)
    w[c] = tot > 0 ? (float)((double)a[c] * a[c] * nchunk / tot) : 0.f;
}

__global__ void k_scale_params(int64_t n, float s, float *__restrict__ w, bf16 *__restrict__ wb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    w[i] *= s;
    wb[i] = __float2bfloat16(w[i]);
  }
}

__global__ void k_f2b(int64_t n, const float *__restrict__ a, bf16 *__restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// parameter offsets in the packed vector: W1 b1 W2 b2 W3 b3
constexpr size_t OW1 = 0, OB1 = OW1 + (size_t)D1 * D0, OW2 = OB1 + D1, OB2 = OW2 + (size_t)D2 * D1,
                 OW3 = OB2 + D2, OB3 = OW3 + (size_t)D3 * D2, NPAR = OB3 + D3;

inline int g1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

// ------------------------------------------------------------------ network state
struct NnState {
  bool ready = false;    // correction enabled (trained and accepted by the validation gate, or set)
  bool trained = false;
  double *dots = nullptr;
  int nchunk = 0;
  int *d_cstart = nullptr, *d_clen = nullptr;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // FP32 master, Adam moments, gradient
  float *splitk = nullptr;  // partial tiles of split-K products
  size_t splitk_cap = 0;
  bf16 *wb = nullptr;                                             // BF16 weights
  int cap = 0;                                                    // activation capacity (samples)
  bf16 *X = nullptr, *H1 = nullptr, *H2 = nullptr;
  float *Y = nullptr, *dY = nullptr, *dH1 = nullptr, *dH2 = nullptr, *nrm = nullptr, *wts = nullptr;
  double *loss = nullptr;
};

static NnState &nn(sie_ctx *c) {
  if (!c->nn) c->nn = new NnState();
  return *(NnState *)c->nn;
}

void nn_free(sie_ctx *c) { delete (NnState *)c->nn; }

static void nn_alloc(sie_ctx *c, int cap) {
  NnState &S = nn(c);
  if (!S.w) {
    // chunks: each global leaf box split into runs of <= 32 bases (internal order)
    std::vector<int> cs, cl;
    for (size_t b = 0; b + 1 < c->leaf_start.size(); ++b)
      for (int s = c->leaf_start[b]; s < c->leaf_start[b + 1]; s += CH) {
        cs.push_back(s);
        cl.push_back(std::min(CH, c->leaf_start[b + 1] - s));
      }
    S.nchunk = (int)cs.size();
    S.d_cstart = dev_upload(c, cs);
    S.d_clen = dev_upload(c, cl);
    S.w = (float *)dev_alloc(c, NPAR * 4);
    S.m = (float *)dev_alloc(c, NPAR * 4);
    S.v = (float *)dev_alloc(c, NPAR * 4);
    S.g = (float *)dev_alloc(c, NPAR * 4);
    S.wb = (bf16 *)dev_alloc(c, NPAR * 2);
    S.loss = (double *)dev_alloc(c, sizeof(double));
    S.dots = (double *)dev_alloc(c, 3 * sizeof(double));
  }
  cap = std::max(cap, S.nchunk);
  if (cap > S.cap) {
    S.X = (bf16 *)dev_alloc(c, (size_t)cap * D0 * 2);
    S.H1 = (bf16 *)dev_alloc(c, (size_t)cap * D1 * 2);
    S.H2 = (bf16 *)dev_alloc(c, (size_t)cap * D2 * 2);
    S.Y = (float *)dev_alloc(c, (size_t)cap * D3 * 4);
    S.dY = (float *)dev_alloc(c, (size_t)cap * D3 * 4);
    S.dH1 = (float *)dev_alloc(c, (size_t)cap * D1 * 4);
    S.dH2 = (float *)dev_alloc(c, (size_t)cap * D2 * 4);
    S.nrm = (float *)dev_alloc(c, (size_t)cap * 4);
    S.wts = (float *)dev_alloc(c, (size_t)cap * 4);
    S.cap = cap;
  }
}

template <typename TA, typename TB>
static void dense(sie_ctx *c, int M, int N, int K, const TA *A, int lda, int ta, const TB *B, int ldb, int tb,
                  const float *bias, int relu, float *Cf, bf16 *Cb) {
  // the forward layers (BF16 activations times BF16 weights, both K-major) on
  // the tensor cores; the gradient products (FP32 factors) on the SIMT tiles
  if (std::is_same<TA, bf16>::value && std::is_same<TB, bf16>::value && !ta && tb && lda == K && ldb == K &&
      nn_dense_tc(c, M, N, K, A, B, bias, relu, Cf, Cb))
    return;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  // a long inner dimension on few output tiles (the weight gradients, summed
  // over the samples): split K so that the GPU fills, slices added in order
  const int tiles = (int)(grid.x * grid.y);
  int S = 1;
  if (K >= 1024 && tiles < 152) S = std::min((K + 255) / 256, std::max(1, (4 * 152) / tiles));
  NnState &St = nn(c);
  if (S > 1 && St.splitk_cap < (size_t)S * M * N) {
    St.splitk = (float *)dev_alloc(c, (size_t)S * M * N * sizeof(float));
    St.splitk_cap = (size_t)S * M * N;
  }
  if (S > 1) {
    const int kch = ((K + S - 1) / S + 15) / 16 * 16;
    S = (K + kch - 1) / kch;
    grid.z = S;
    k_dense<TA, TB><<<grid, 256, 0, c->stream>>>(M, N, K, kch, A, lda, ta, B, ldb, tb, bias, relu, St.splitk, Cb);
    SIE_CHECK_LAUNCH();
    const int64_t mn = (int64_t)M * N;
    k_splitk_sum<<<(unsigned)((mn + 255) / 256), 256, 0, c->stream>>>(mn, N, S, St.splitk, bias, relu, Cf, Cb);
    SIE_CHECK_LAUNCH();
    c->launches += 2;
    return;
  }
  k_dense<TA, TB><<<grid, 256, 0, c->stream>>>(M, N, K, K, A, lda, ta, B, ldb, tb, bias, relu, Cf, Cb);
  SIE_CHECK_LAUNCH();
  c->launches++;
}

// forward of n samples whose inputs are in S.X[off..]; output FP32 in S.Y
static void nn_forward(sie_ctx *c, NnState &S, int n, size_t off) {
  const bf16 *X = S.X + off * D0;
  dense(c, n, D1, D0, X, D0, 0, S.wb + OW1, D0, 1, S.w + OB1, 1, (float *)nullptr, S.H1 + off * D1);
  dense(c, n, D2, D1, S.H1 + off * D1, D1, 0, S.wb + OW2, D1, 1, S.w + OB2, 1, (float *)nullptr, S.H2 + off * D2);
  dense(c, n, D3, D2, S.H2 + off * D2, D2, 0, S.wb + OW3, D2, 1, S.w + OB3, 0, S.Y + off * D3, (bf16 *)nullptr);
}

// gradient of the (weighted, wt may be null) MSE loss over samples [off, off+n)
// against targets T -> S.g; the loss is added to S.loss
static void nn_backward(sie_ctx *c, NnState &S, int n, size_t off, const float *T, const float *wt) {
  const float inv_n = 1.f / (float)n;
  k_mse<<<g1((int64_t)n * D3), 256, 0, c->stream>>>((int64_t)n * D3, inv_n, S.Y + off * D3, T + off * D3,
                                                    wt ? wt + off : nullptr, S.dY + off * D3, S.loss);
  SIE_CHECK_LAUNCH();
  const float *dY = S.dY + off * D3;
  const bf16 *X = S.X + off * D0, *H1 = S.H1 + off * D1, *H2 = S.H2 + off * D2;
  // layer 3
  dense(c, D3, D2, n, dY, D3, 1, H2, D2, 0, (const float *)nullptr, 0, S.g + OW3, (bf16 *)nullptr);
  k_colsum<<<1, D3, 0, c->stream>>>(n, D3, dY, S.g + OB3);
  dense(c, n, D2, D3, dY, D3, 0, S.wb + OW3, D2, 0, (const float *)nullptr, 0, S.dH2 + off * D2, (bf16 *)nullptr);
  k_relu_mask<<<g1((int64_t)n * D2), 256, 0, c->stream>>>((int64_t)n * D2, H2, S.dH2 + off * D2);
  // layer 2
  dense(c, D2, D1, n, S.dH2 + off * D2, D2, 1, H1, D1, 0, (const float *)nullptr, 0, S.g + OW2, (bf16 *)nullptr);
  k_colsum<<<1, D2, 0, c->stream>>>(n, D2, S.dH2 + off * D2, S.g + OB2);
  dense(c, n, D1, D2, S.dH2 + off * D2, D2, 0, S.wb + OW2, D1, 0, (const float *)nullptr, 0, S.dH1 + off * D1,
        (bf16 *)nullptr);
  k_relu_mask<<<g1((int64_t)n * D1), 256, 0, c->stream>>>((int64_t)n * D1, H1, S.dH1 + off * D1);
  // layer 1
  dense(c, D1, D0, n, S.dH1 + off * D1, D1, 1, X, D0, 0, (const float *)nullptr, 0, S.g + OW1, (bf16 *)nullptr);
  k_colsum<<<1, D1, 0, c->stream>>>(n, D1, S.dH1 + off * D1, S.g + OB1);
  SIE_CHECK_LAUNCH();
  c->launches += 5;
}

// ------------------------------------------------------------------ used by the solver
bool nn_ready(sie_ctx *c) { return c->nn && ((NnState *)c->nn)->ready; }
bool nn_trained(sie_ctx *c) { return c->nn && (((NnState *)c->nn)->trained || ((NnState *)c->nn)->ready); }

// z (internal order, FP64) += chunk-wise network correction computed from v
void nn_apply(sie_ctx *c, const zd *v, zd *z, int nrhs) {
  NnState &S = nn(c);
  const int ne2 = 2 * c->ne;
  for (int r = 0; r < nrhs; ++r) {
    // input: the ILU(0) output already in z (u = ILU^-1 v), chunk by chunk
    (void)v;
    k_chunk_gather<<<S.nchunk, 128, 0, c->stream>>>(S.nchunk, S.d_cstart, S.d_clen, z + (size_t)r * ne2, S.X, S.nrm);
    SIE_CHECK_LAUNCH();
    nn_forward(c, S, S.nchunk, 0);
    k_chunk_scatter<<<S.nchunk, 64, 0, c->stream>>>(S.nchunk, S.d_cstart, S.d_clen, S.Y, S.nrm, z + (size_t)r * ne2);
    SIE_CHECK_LAUNCH();
    c->launches += 2;
  }
}

// ------------------------------------------------------------------ API
extern "C" sie_status nnprec_train(sie_ctx *c, const sie_nn_opts *o, sie_nn_stats *st) {
  if (!c) return SIE_EINVAL;
  try {
    SIE_CUDA(cudaSetDevice(c->device));
    SIE_REQUIRE(c->have_fill && c->ilu.ready, SIE_ESTATE, "nnprec_train: needs the near field and ILU factors");
    SIE_REQUIRE(o && st && o->ntrain >= 1 && o->train_inc && o->epochs >= 1 && o->batch >= 64 && o->lr > 0 &&
                    o->record_restart >= 1,
                SIE_EINVAL, "nnprec_train: bad options");
    cudaEvent_t e0, e1;
    SIE_CUDA(cudaEventCreate(&e0));
    SIE_CUDA(cudaEventCreate(&e1));
    SIE_CUDA(cudaEventRecord(e0, c->stream));
    nn_alloc(c, 0);
    NnState &S = nn(c);
    S.ready = false;
    const int ne = c->ne, ne2 = 2 * ne;
    // 1. pairs recorded by the solver: restarts of FGMRES(record_restart) with ILU(0)
    std::vector<zd *> R, E;
    int cap_pairs = std::max(1, o->max_pairs);
    ensure_work(c, 1);
    zd *b = (zd *)dev_alloc(c, (size_t)ne2 * sizeof(zd));
    zd *rec_x = (zd *)dev_alloc(c, (size_t)cap_pairs * ne2 * sizeof(zd));
    zd *rec_r = (zd *)dev_alloc(c, (size_t)cap_pairs * ne2 * sizeof(zd));
    zd *xs = (zd *)dev_alloc(c, (size_t)ne2 * sizeof(zd));
    zd *zilu = (zd *)dev_alloc(c, (size_t)ne2 * sizeof(zd));
    double *d_inc = (double *)stage(c, 4 * sizeof(double));
    int npairs = 0;
    std::vector<int> owner;  // training solve of each pair
    for (int t = 0; t < o->ntrain && npairs < cap_pairs; ++t) {
      SIE_CUDA(cudaMemcpyAsync(d_inc, o->train_inc + 4 * t, 4 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      launch_rhs(c, d_inc, 1, b);  // internal order
      SIE_CUDA(cudaMemsetAsync(xs, 0, (size_t)ne2 * sizeof(zd), c->stream));
      int first = npairs;
      Recorder rec{rec_x, rec_r, cap_pairs, &npairs};
      run_gmres_internal(c, b, xs, 1, o->record_restart, 1000, 1e-7, SIE_PREC_MIXED,
                         residual_prec(SIE_PREC_MIXED, 1e-7, false), 1, &rec, nullptr);
      for (int k = first; k < npairs; ++k) owner.push_back(t);
      // errors e_k = x* - x_k (stored over rec_x)
      for (int k = first; k < npairs; ++k) {
        zd *xk = rec_x + (size_t)k * ne2;
        op_sub(c, xs, xk, xk, (int64_t)ne2);  // xk <- xs - xk
      }
    }
    SIE_REQUIRE(npairs > 0, SIE_EINVAL, "nnprec_train: the recording solves produced no pairs");
    // 2. samples: per pair and chunk, u = ILU^-1 r, input u_c / |u_c|, target (e - u)_c / |u_c|
    const int64_t nsamp = (int64_t)npairs * S.nchunk;
    SIE_REQUIRE(nsamp < (1LL << 31) / D1, SIE_EINVAL, "nnprec_train: too many samples");
    nn_alloc(c, (int)nsamp);
    float *T = (float *)dev_alloc(c, (size_t)nsamp * D3 * sizeof(float));
    for (int k = 0; k < npairs; ++k) {
      zd *rk = rec_r + (size_t)k * ne2, *ek = rec_x + (size_t)k * ne2;
      apply_ilu(c, rk, zilu, 1, SIE_PREC_FP64);
      k_chunk_gather<<<S.nchunk, 128, 0, c->stream>>>(S.nchunk, S.d_cstart, S.d_clen, zilu,
                                                      S.X + (size_t)k * S.nchunk * D0, S.nrm + (size_t)k * S.nchunk);
      k_chunk_target<<<S.nchunk, 128, 0, c->stream>>>(S.nchunk, S.d_cstart, S.d_clen, ek, zilu,
                                                      S.nrm + (size_t)k * S.nchunk, T + (size_t)k * S.nchunk * D3);
      SIE_CHECK_LAUNCH();
      c->launches += 2;
    }
    // sample weights |u_c|^2 (normalised per pair): the loss is the error of z itself
    k_pair_weights<<<npairs, 256, 0, c->stream>>>(S.nchunk, S.nrm, S.wts);
    SIE_CHECK_LAUNCH();
    c->launches++;
    // 3. initialise (He, seeded) and train with Adam on shuffled minibatches of whole sample blocks
    std::mt19937_64 rng(o->seed);
    std::vector<float> w(NPAR, 0.f);
    auto init = [&](size_t off, int fan_in, int fan_out, float scale) {
      std::normal_distribution<float> nd(0.f, scale * std::sqrt(2.f / fan_in));
      for (size_t i = 0; i < (size_t)fan_in * fan_out; ++i) w[off + i] = nd(rng);
    };
    init(OW1, D0, D1, 1.f);
    init(OW2, D1, D2, 1.f);
    init(OW3, D2, D3, 0.1f);  // start close to the plain ILU preconditioner
    SIE_CUDA(cudaMemcpyAsync(S.w, w.data(), NPAR * 4, cudaMemcpyHostToDevice, c->stream));
    SIE_CUDA(cudaMemsetAsync(S.m, 0, NPAR * 4, c->stream));
    SIE_CUDA(cudaMemsetAsync(S.v, 0, NPAR * 4, c->stream));
    k_f2b<<<g1(NPAR), 256, 0, c->stream>>>((int64_t)NPAR, S.w, S.wb);
    SIE_CHECK_LAUNCH();
    // hold out the pairs of the last fifth of the incidences (at least one when
    // there are two or more) for the validation gate
    const int nval_inc = o->ntrain >= 2 ? std::max(1, o->ntrain / 5) : 0;
    int nval = 0;
    for (int k = 0; k < npairs; ++k)
      if (owner[k] >= o->ntrain - nval_inc) ++nval;
    if (nval == npairs) nval = 0;
    const int64_t ntr_s = (int64_t)(npairs - nval) * S.nchunk;
    const int B = std::min<int64_t>(o->batch, ntr_s);
    const int nbat = (int)((ntr_s + B - 1) / B);
    int step = 0;
    double loss_first = -1, loss_last = 0;
    std::vector<int> order(nbat);
    for (int i = 0; i < nbat; ++i) order[i] = i;
    for (int ep = 0; ep < o->epochs; ++ep) {
      std::shuffle(order.begin(), order.end(), rng);
      SIE_CUDA(cudaMemsetAsync(S.loss, 0, sizeof(double), c->stream));
      for (int bi : order) {
        size_t off = (size_t)bi * B;
        int n = (int)std::min<int64_t>(B, ntr_s - (int64_t)off);
        nn_forward(c, S, n, off);
        nn_backward(c, S, n, off, T, S.wts);
        ++step;
        float c1 = 1.f - std::pow(0.9f, (float)step), c2 = 1.f - std::pow(0.999f, (float)step);
        k_adam<<<g1(NPAR), 256, 0, c->stream>>>((int64_t)NPAR, (float)o->lr, 0.9f, 0.999f, 1e-8f, c1, c2, S.g, S.w,
                                                S.m, S.v, S.wb);
        SIE_CHECK_LAUNCH();
        c->launches++;
      }
      double l = 0;
      SIE_CUDA(cudaMemcpyAsync(&l, S.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      SIE_CUDA(cudaStreamSynchronize(c->stream));
      l /= nbat;
      if (loss_first < 0) loss_first = l;
      loss_last = l;
    }
    SIE_CUDA(cudaEventRecord(e1, c->stream));
    SIE_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    SIE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // validation gate: best output scale g* = <Y,T>/<Y,Y> on held-out samples;
    // the correction is kept (scaled by min(g*, 1)) only if it lowers the
    // held-out loss below 95 % of the loss of no correction at all
    const int64_t v0 = nval ? ntr_s : 0, nv = nval ? nsamp - ntr_s : ntr_s;
    SIE_CUDA(cudaMemsetAsync(S.dots, 0, 3 * sizeof(double), c->stream));
    for (int64_t off = v0; off < v0 + nv; off += B) {
      int n = (int)std::min<int64_t>(B, v0 + nv - off);
      nn_forward(c, S, n, (size_t)off);
      k_dots<<<g1((int64_t)n * D3), 256, 0, c->stream>>>((int64_t)n * D3, S.Y + (size_t)off * D3,
                                                        T + (size_t)off * D3, S.wts + off, S.dots);
      SIE_CHECK_LAUNCH();
      c->launches++;
    }
    double dots[3];
    SIE_CUDA(cudaMemcpyAsync(dots, S.dots, sizeof(dots), cudaMemcpyDeviceToHost, c->stream));
    SIE_CUDA(cudaStreamSynchronize(c->stream));
    double gam = dots[1] > 0 ? dots[0] / dots[1] : 0.0;
    double ratio = dots[2] > 0 ? 1.0 - (dots[1] > 0 ? dots[0] * dots[0] / (dots[1] * dots[2]) : 0.0) : 1.0;
    bool enabled = gam > 0 && ratio < 0.95;
    if (enabled) {
      float sc = (float)std::min(gam, 1.0);
      k_scale_params<<<g1((int64_t)(NPAR - OW3)), 256, 0, c->stream>>>((int64_t)(NPAR - OW3), sc, S.w + OW3, S.wb + OW3);
      SIE_CHECK_LAUNCH();
      SIE_CUDA(cudaStreamSynchronize(c->stream));
    }
    // the plain ILU(0) solver decides: solve the last (held-out) incidence
    // with and without the correction; keep it only if it saves iterations
    int it_ilu = -1, it_nn = -1;
    if (enabled) {
      SIE_CUDA(cudaMemcpyAsync(d_inc, o->train_inc + 4 * (o->ntrain - 1), 4 * sizeof(double), cudaMemcpyHostToDevice,
                               c->stream));
      launch_rhs(c, d_inc, 1, b);
      sie_solve_stats sv;
      S.ready = false;
      SIE_CUDA(cudaMemsetAsync(xs, 0, (size_t)ne2 * sizeof(zd), c->stream));
      run_gmres_internal(c, b, xs, 1, 50, 1000, 1e-4, SIE_PREC_MIXED, residual_prec(SIE_PREC_MIXED, 1e-4, false),
                         1, nullptr, &sv);
      it_ilu = sv.iters;
      S.ready = true;
      SIE_CUDA(cudaMemsetAsync(xs, 0, (size_t)ne2 * sizeof(zd), c->stream));
      run_gmres_internal(c, b, xs, 1, 50, 1000, 1e-4, SIE_PREC_MIXED, residual_prec(SIE_PREC_MIXED, 1e-4, false),
                         2, nullptr, &sv);
      it_nn = sv.iters;
      enabled = it_nn < it_ilu;
    }
    st->gate_iters_ilu = it_ilu;
    st->gate_iters_nn = it_nn;
    S.trained = true;
    S.ready = enabled;
    st->val_loss_ratio = ratio;
    st->gamma = gam;
    st->enabled = enabled ? 1 : 0;
    st->pairs = npairs;
    st->samples = nsamp;
    st->loss_first = loss_first;
    st->loss_last = loss_last;
    st->ms = ms;
    return SIE_OK;
  } catch (const SieError &e) {
    c->last_error = e.msg;
    return e.code;
  } catch (const std::exception &e) {
    c->last_error = e.what();
    return SIE_EINVAL;
  }
}

extern "C" sie_status nnprec_params(sie_ctx *c, float *params, int32_t set) {
  if (!c || !params) return SIE_EINVAL;
  try {
    SIE_CUDA(cudaSetDevice(c->device));
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "nnprec_params: call sie_fill_nearfield first");
    nn_alloc(c, 0);
    NnState &S = nn(c);
    if (set) {
      SIE_CUDA(cudaMemcpyAsync(S.w, params, NPAR * 4, cudaMemcpyHostToDevice, c->stream));
      k_f2b<<<g1(NPAR), 256, 0, c->stream>>>((int64_t)NPAR, S.w, S.wb);
      SIE_CHECK_LAUNCH();
      S.ready = true;
      S.trained = true;
    } else {
      SIE_CUDA(cudaMemcpyAsync(params, S.w, NPAR * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    SIE_CUDA(cudaStreamSynchronize(c->stream));
    return SIE_OK;
  } catch (const SieError &e) {
    c->last_error = e.msg;
    return e.code;
  }
}

extern "C" sie_status nnprec_loss_grad(sie_ctx *c, const float *X_host, const float *T_host, int64_t n,
                                       double *loss, float *grad_host) {
  if (!c || !X_host || !T_host || !loss || !grad_host || n < 1) return SIE_EINVAL;
  try {
    SIE_CUDA(cudaSetDevice(c->device));
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "nnprec_loss_grad: call sie_fill_nearfield first");
    SIE_REQUIRE(n <= (1 << 20), SIE_EINVAL, "nnprec_loss_grad: at most 2^20 samples");
    nn_alloc(c, (int)n);
    NnState &S = nn(c);
    float *Xf = (float *)stage(c, (size_t)n * (D0 + D3) * sizeof(float));
    float *Tf = Xf + (size_t)n * D0;
    SIE_CUDA(cudaMemcpyAsync(Xf, X_host, (size_t)n * D0 * 4, cudaMemcpyHostToDevice, c->stream));
    SIE_CUDA(cudaMemcpyAsync(Tf, T_host, (size_t)n * D3 * 4, cudaMemcpyHostToDevice, c->stream));
    k_f2b<<<g1((int64_t)n * D0), 256, 0, c->stream>>>((int64_t)n * D0, Xf, S.X);
    SIE_CHECK_LAUNCH();
    SIE_CUDA(cudaMemsetAsync(S.loss, 0, sizeof(double), c->stream));
    nn_forward(c, S, (int)n, 0);
    nn_backward(c, S, (int)n, 0, Tf, nullptr);
    SIE_CUDA(cudaMemcpyAsync(grad_host, S.g, NPAR * 4, cudaMemcpyDeviceToHost, c->stream));
    SIE_CUDA(cudaMemcpyAsync(loss, S.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SIE_CUDA(cudaStreamSynchronize(c->stream));
    return SIE_OK;
  } catch (const SieError &e) {
    c->last_error = e.msg;
    return e.code;
  }
}
