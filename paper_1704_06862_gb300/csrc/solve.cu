// Restarted flexible GMRES with right preconditioning for a block of
// independent right-hand sides run in lockstep.  Arnoldi vectors, classical
// Gram-Schmidt with one re-orthogonalisation, and the true residual at every
// restart are FP64 on the device; the Hessenberg least-squares problem (Givens
// rotations) is solved on the host.  With SIE_PREC_MIXED the inner operator
// and preconditioner run in FP32 while the restart residual is recomputed in
// FP64 vectors with the FP64 near field (SIE_PREC_NEAR64: far field in FP32,
// added into the FP64 product; or the whole FP64 operator on request), which
// makes the restarts an iterative refinement.
#include <algorithm>
#include <cmath>
#include <complex>

#include "common.h"

namespace {

typedef std::complex<double> cd;

// Square root of a computed sum of squares: a rounding below zero gives 0, a
// NaN stays NaN (a non-finite vector must reach the solvers' breakdown checks;
// std::max(0.0, NaN) would turn it into a zero norm and a false convergence).
inline double sqrt_nonneg(double v) { return std::isnan(v) ? v : std::sqrt(v > 0.0 ? v : 0.0); }

// Two-stage dot products h[i][r] = sum_n conj(V_i[r][n]) w[r][n], i < nvec.
// Stage 1: one warp per (vector i, chunk of ch elements, rhs r), lanes over
// the chunk with four independent accumulators (the FP64 multiply-adds of
// this GPU are few and long: independent chains keep them busy), one partial
// per warp (no block-level synchronisation); stage 2 adds the partials in
// chunk order.  Chunks of MD_CH elements for several vectors, MD_CH1 for a
// single one (a norm), so that either fills the GPU.  With a gate,
// right-hand sides whose gate is 0 get zero partials.
constexpr int MD_CH = 1024, MD_CH1 = 256;
// Gram-Schmidt kernels chained by programmatic dependent launch (each waits
// for its predecessor first thing: stream order, launch latency hidden)
constexpr bool GS_CHAINED = true;
__global__ void __launch_bounds__(256) k_mdot_part(int n, int nrhs, int nvec, int nblk, int ch,
                                                  const zd *__restrict__ V, size_t vstride,
                                                  const zd *__restrict__ w, zd *__restrict__ part,
                                                  const int *__restrict__ gate) {
  pdl_wait();
  pdl_release();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r = blockIdx.y;
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
  if (gw >= nvec * nblk) return;
  const int i = gw / nblk, blk = gw - i * nblk;
  zd acc;
  if (!gate || gate[r]) {
    const zd *a = V + (size_t)i * vstride + (size_t)r * n;
    const zd *x = w + (size_t)r * n;
    const int t1 = min(n, (blk + 1) * ch);
    zd a1, a2, a3;
    int t = blk * ch + lane;
#pragma unroll 2
    for (; t + 96 < t1; t += 128) {
      acc = cfma(conj(a[t]), x[t], acc);
      a1 = cfma(conj(a[t + 32]), x[t + 32], a1);
      a2 = cfma(conj(a[t + 64]), x[t + 64], a2);
      a3 = cfma(conj(a[t + 96]), x[t + 96], a3);
    }
    for (; t < t1; t += 32) acc = cfma(conj(a[t]), x[t], acc);
    acc = (acc + a1) + (a2 + a3);
    for (int d = 16; d > 0; d >>= 1) {
      acc.re += __shfl_down_sync(0xffffffffu, acc.re, d);
      acc.im += __shfl_down_sync(0xffffffffu, acc.im, d);
    }
  }
  if (lane == 0) part[((size_t)i * nrhs + r) * nblk + blk] = acc;
}

__global__ void k_mdot_sum(int nrhs, int nblk, const zd *__restrict__ part, zd *__restrict__ h) {
  pdl_wait();
  pdl_release();
  const int i = blockIdx.x, r = blockIdx.y;
  __shared__ double2 red_raw[256];  // raw storage: zd has a constructor
  zd *red = reinterpret_cast<zd *>(red_raw);
  zd acc;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[((size_t)i * nrhs + r) * nblk + b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) h[(size_t)i * nrhs + r] = red[0];
}

// One classical Gram-Schmidt update fused with the norm that follows it:
//   w[r] -= sum_{i<j1} V_i[r] h[i][r]   (unless gate_in is given and gate_in[r] == 0),
//   nn[r] = |w[r]|^2,
// and with gate_out the selective second-pass test (Daniel-Gragg-Kaufman-
// Stewart): after the first pass |w|^2 = |w'|^2 + |h|^2, and the pass is
// repeated only when |w'| < |w| / sqrt(2), i.e. |w'|^2 < |h|^2.  Each CTA adds its squares in a fixed order and writes one
// partial; the last CTA to finish (a counter, reset by that CTA) adds the
// partials in CTA order, one warp per right-hand side: deterministic, and one
// launch instead of three.
__global__ void __launch_bounds__(256) k_orth_norm(int n, int nrhs, int j1, const zd *__restrict__ V, size_t vstride,
                                                  const zd *__restrict__ h, zd *__restrict__ w,
                                                  const int *__restrict__ gate_in, double *__restrict__ npart,
                                                  unsigned *__restrict__ cnt, zd *__restrict__ nn,
                                                  int *__restrict__ gate_out) {
  pdl_wait();
  pdl_release();
  const int t = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double sq = 0.0;
  if (t < n) {
    zd x = w[(size_t)r * n + t];
    if (!gate_in || gate_in[r]) {
      const zd *v = V + (size_t)r * n + t;
      zd a0, a1, a2, a3;
      int i = 0;
#pragma unroll 2
      for (; i + 3 < j1; i += 4) {
        a0 += v[(size_t)i * vstride] * h[(size_t)i * nrhs + r];
        a1 += v[(size_t)(i + 1) * vstride] * h[(size_t)(i + 1) * nrhs + r];
        a2 += v[(size_t)(i + 2) * vstride] * h[(size_t)(i + 2) * nrhs + r];
        a3 += v[(size_t)(i + 3) * vstride] * h[(size_t)(i + 3) * nrhs + r];
      }
      for (; i < j1; ++i) a0 += v[(size_t)i * vstride] * h[(size_t)i * nrhs + r];
      x = x - ((a0 + a1) + (a2 + a3));
      w[(size_t)r * n + t] = x;
    }
    sq = x.re * x.re + x.im * x.im;
  }
  for (int d = 16; d > 0; d >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, d);
  __shared__ double red[8];
  __shared__ int s_last;
  if (lane == 0) red[warp] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b += red[k];
    npart[(size_t)r * gridDim.x + blockIdx.x] = b;
    __threadfence();
    const unsigned prev = atomicAdd(cnt, 1u);
    s_last = prev == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int rr = warp; rr < nrhs; rr += (int)(blockDim.x >> 5)) {
    double a = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(npart + (size_t)rr * gridDim.x + b);
    for (int d = 16; d > 0; d >>= 1) a += __shfl_down_sync(0xffffffffu, a, d);
    if (lane == 0) {
      nn[rr] = zd(a, 0.0);
      if (gate_out) {
        double hh = 0.0;
        for (int i = 0; i < j1; ++i) {
          const zd v = h[(size_t)i * nrhs + rr];
          hh += v.re * v.re + v.im * v.im;
        }
        gate_out[rr] = a < hh ? 1 : 0;
      }
    }
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

// out[r] = a[r] * s[r]
__global__ void k_scale(int n, const zd *__restrict__ a, const zd *__restrict__ s, zd *__restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (t >= n) return;
  out[(size_t)r * n + t] = a[(size_t)r * n + t] * s[r];
}

// V_{j+1}[r] = w[r] / sqrt(nn[r]) where nn[r] = <w[r], w[r]>; zero for right-hand
// sides that are finished (act[r] == 0) or whose new vector vanished
__global__ void k_scale_norm(int n, const zd *__restrict__ a, const zd *__restrict__ nn, const zd *__restrict__ act,
                             zd *__restrict__ out) {
  pdl_wait();
  pdl_release();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (t >= n) return;
  const double q = nn[r].re;
  const double s = (act[r].re != 0.0 && q > 0.0) ? 1.0 / sqrt(q) : 0.0;
  out[(size_t)r * n + t] = a[(size_t)r * n + t] * s;
}

// out = a - b
__global__ void k_sub(int64_t n, const zd *a, const zd *b, zd *out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = a[t] - b[t];
}

// out[r] = a[r] + c[r] b[r]   (per right-hand-side complex coefficient)
__global__ void k_axpy_r(int n, const zd *__restrict__ a, const zd *__restrict__ cf, const zd *__restrict__ b,
                         zd *__restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (t >= n) return;
  const size_t i = (size_t)r * n + t;
  out[i] = a[i] + cf[r] * b[i];
}
// out[r] = a[r] + c1[r] (b[r] + c2[r] d[r])
__global__ void k_axpy2_r(int n, const zd *__restrict__ a, const zd *__restrict__ c1, const zd *__restrict__ b,
                          const zd *__restrict__ c2, const zd *__restrict__ d, zd *__restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (t >= n) return;
  const size_t i = (size_t)r * n + t;
  out[i] = a[i] + c1[r] * (b[i] + c2[r] * d[i]);
}

// x[r] += sum_j Z_j[r] y[j][r]
__global__ void k_xupd(int n, int nrhs, int m, const zd *__restrict__ Z, size_t zstride, const zd *__restrict__ y,
                       zd *__restrict__ x) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (t >= n) return;
  zd acc = x[(size_t)r * n + t];
#pragma unroll 8
  for (int j = 0; j < m; ++j) acc += Z[(size_t)j * zstride + (size_t)r * n + t] * y[(size_t)j * nrhs + r];
  x[(size_t)r * n + t] = acc;
}

struct Gm {
  sie_ctx *c;
  int n, R;
  int nblk;
  zd *part;
  void launch_check() {
    SIE_CHECK_LAUNCH();
    c->launches++;
  }
  // h[i][r] = <V_i[r], w[r]> for i < nvec
  void mdot(const zd *V, size_t vstride, int nvec, const zd *w, zd *d_h, const int *gate = nullptr) {
    // a single vector (a norm) in finer chunks; the partial buffer holds
    // 4 nvec_max R chunks of MD_CH elements, enough for either
    const int ch = nvec == 1 ? MD_CH1 : MD_CH, nb = std::max(1, (n + ch - 1) / ch);
    SIE_CUDA(launch_chained(GS_CHAINED, k_mdot_part, dim3((nvec * nb + 7) / 8, R), dim3(256), 0, c->stream, n, R, nvec,
                            nb, ch, V, vstride, w, part, gate));
    launch_check();
    SIE_CUDA(launch_chained(GS_CHAINED, k_mdot_sum, dim3(nvec, R), dim3(256), 0, c->stream, R, nb, (const zd *)part,
                            d_h));
    launch_check();
  }
  void norms(const zd *w, zd *d_h, std::vector<double> &out) {
    mdot(w, 0, 1, w, d_h);
    std::vector<zd> h(R);
    SIE_CUDA(cudaMemcpyAsync(h.data(), d_h, R * sizeof(zd), cudaMemcpyDeviceToHost, c->stream));
    SIE_CUDA(cudaStreamSynchronize(c->stream));
    out.resize(R);
    for (int r = 0; r < R; ++r) out[r] = sqrt_nonneg(h[r].re);
  }
};

// One CUDA graph per Krylov step index j holding "preconditioner, then
// product" on that step's fixed vectors (V_j, Z_j, w), captured on first use
// and replayed on later iterations and solves of the same shape; invalidated
// when any work buffer is reallocated.  If capture is not possible (the
// stream is already capturing, or capture fails) the step runs eagerly.
struct StepGraphs {
  int m = -1, R = -1, prec = -1, precond = -1;
  int64_t gen = -1;
  bool ok = true;
  std::vector<cudaGraphExec_t> ex;
  std::vector<int64_t> nk;  // kernels per graph (launch accounting)
  void clear() {
    for (auto e : ex)
      if (e) cudaGraphExecDestroy(e);
    ex.clear();
    nk.clear();
  }
  template <typename F>
  void run(sie_ctx *c, int j, F &&step) {
    if (ok && !c->graphs_off && !ex[j]) {
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
          cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        ok = false;
      } else {
        int64_t l0 = c->launches;
        bool fail = false;
        try {
          step();
        } catch (...) {
          fail = true;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        cudaGraphExec_t x = nullptr;
        if (!fail && e == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
          ex[j] = x;
          nk[j] = c->launches - l0;
        } else {
          ok = false;
          cudaGetLastError();
        }
        if (g) cudaGraphDestroy(g);
        c->launches = l0;
      }
    }
    if (ok && !c->graphs_off && ex[j]) {
      SIE_CUDA(cudaGraphLaunch(ex[j], c->stream));
      c->launches += nk[j];
    } else {
      step();
    }
  }
};

StepGraphs &step_graphs(sie_ctx *c, int m, int R, sie_prec prec, int precond) {
  if (!c->graphs) c->graphs = new StepGraphs();
  StepGraphs &G = *(StepGraphs *)c->graphs;
  if (G.m != m || G.R != R || G.prec != (int)prec || G.precond != precond || G.gen != c->work_gen) {
    G.clear();
    G.m = m;
    G.R = R;
    G.prec = (int)prec;
    G.precond = precond;
    G.gen = c->work_gen;
    G.ok = true;
    G.ex.assign(m, nullptr);
    G.nk.assign(m, 0);
  }
  return G;
}

}  // namespace

int graphs_state(const sie_ctx *c) {
  if (!c->graphs) return -1;
  const StepGraphs &G = *(const StepGraphs *)c->graphs;
  if (!G.ok) return 0;
  for (auto e : G.ex)
    if (e) return 1;
  return -1;
}

void graphs_free(sie_ctx *c) {
  if (!c->graphs) return;
  StepGraphs *G = (StepGraphs *)c->graphs;
  G->clear();
  delete G;
  c->graphs = nullptr;
}

// Restarted FGMRES on internal-order FP64 vectors b, x (x holds the initial
// guess).  precond: 0 none, 1 ILU(0), 2 ILU(0) followed by the learned
// correction; the learned part is switched off for the rest of the solve as
// soon as a restart cycle fails to reduce the true residual.  With a recorder
// (one right-hand side), the iterate and true residual of every restart
// before convergence are copied out as training pairs.
sie_status run_gmres_internal(sie_ctx *c, const zd *b, zd *x, int R, int m, int max_iters, double tol,
                              sie_prec prec, sie_prec rprec, int precond, Recorder *rec, sie_solve_stats *st) {
  const int n = 2 * c->ne;
  const size_t vs = (size_t)R * n;
  ensure_work(c, R);
  // Krylov storage (allocated once per capacity and kept in the context)
  static_assert(sizeof(zd) == 16, "complex layout");
  if (c->gm_m != m || c->gm_R != R) {
    c->gm_V = dev_alloc(c, (size_t)(m + 1) * vs * sizeof(zd));
    c->gm_Z = dev_alloc(c, (size_t)m * vs * sizeof(zd));
    c->gm_w = dev_alloc(c, vs * sizeof(zd));
    c->gm_h = dev_alloc(c, 3 * (size_t)(m + 2) * R * sizeof(zd));  // h (first pass), h (second pass), |w|^2
    c->gm_s = dev_alloc(c, (size_t)(m + 2) * R * sizeof(zd));
    c->gm_act = dev_alloc(c, (size_t)R * sizeof(zd));
    if (c->gm_hpin) cudaFreeHost(c->gm_hpin);
    c->gm_hpin = nullptr;
    SIE_CUDA(cudaMallocHost(&c->gm_hpin, 3 * (size_t)(m + 2) * R * sizeof(zd)));
    if (!c->gm_ev) SIE_CUDA(cudaEventCreateWithFlags(&c->gm_ev, cudaEventDisableTiming));
    c->gm_part = dev_alloc(c, (size_t)std::max(m + 2, 4) * R * ((n + MD_CH - 1) / MD_CH) * sizeof(zd));
    c->gm_gate = dev_alloc(c, (size_t)R * sizeof(int));
    c->gm_npart = dev_alloc(c, (size_t)R * ((n + 255) / 256) * sizeof(double));
    c->gm_cnt = dev_alloc(c, 256);
    SIE_CUDA(cudaMemsetAsync(c->gm_cnt, 0, 256, c->stream));
    if (!c->gm_cs) SIE_CUDA(cudaStreamCreateWithFlags(&c->gm_cs, cudaStreamNonBlocking));
    if (!c->gm_ev0) SIE_CUDA(cudaEventCreateWithFlags(&c->gm_ev0, cudaEventDisableTiming));
    c->gm_m = m;
    c->gm_R = R;
    c->work_gen++;
  }
  zd *V = (zd *)c->gm_V, *Z = (zd *)c->gm_Z, *w = (zd *)c->gm_w;
  StepGraphs &SG = step_graphs(c, m, R, prec, precond);
  zd *d_h = (zd *)c->gm_h, *d_s = (zd *)c->gm_s;
  // 256 threads x 4 elements per block
  Gm g{c, n, R, std::max(1, (n + MD_CH - 1) / MD_CH), (zd *)c->gm_part};  // chunks of MD_CH elements
  bool use_nn = precond == 2 && nn_ready(c);
  std::vector<double> prev_res(R, HUGE_VAL);
  std::vector<double> bn, rn;
  g.norms(b, d_h, bn);
  std::vector<int> iters(R, 0), restarts(R, 0), active(R, 1);
  std::vector<double> relres(R, 0.0);
  dim3 gv((n + 255) / 256, R);
  sie_status status = SIE_OK;
  int total = 0;
  std::vector<cd> H((size_t)(m + 1) * m * R), gvec((size_t)(m + 1) * R), sn((size_t)m * R);
  std::vector<double> cs((size_t)m * R);
  std::vector<double> xn;
  g.norms(x, d_h, xn);
  bool x_zero = true;
  for (int r = 0; r < R; ++r) x_zero = x_zero && xn[r] == 0.0;
  bool first = true;
  for (;;) {
    // true residual with the residual operator rprec (r = b for a zero initial guess)
    if (first && x_zero) {
      SIE_CUDA(cudaMemcpyAsync(w, b, vs * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      apply_matvec(c, x, w, R, rprec, 3);
      k_sub<<<std::min(152 * 16, (int)((vs + 255) / 256)), 256, 0, c->stream>>>((int64_t)vs, b, w, w);
      g.launch_check();
    }
    first = false;
    g.norms(w, d_h, rn);
    check_device_error(c);  // a preconditioner apply whose bounded wait gave up
    bool any = false;
    for (int r = 0; r < R; ++r) {
      relres[r] = bn[r] > 0 ? rn[r] / bn[r] : (std::isnan(bn[r]) ? bn[r] : 0.0);
      if (!std::isfinite(relres[r])) {
        status = SIE_EBREAKDOWN;
        active[r] = 0;
        continue;
      }
      active[r] = relres[r] > tol && iters[r] < max_iters;
      if (active[r]) any = true;
      if (use_nn && rn[r] >= prev_res[r]) use_nn = false;  // fall back to plain ILU(0)
      prev_res[r] = rn[r];
    }
    if (!any || status != SIE_OK) break;
    if (rec && R == 1 && *rec->count < rec->cap) {
      int k = (*rec->count)++;
      SIE_CUDA(cudaMemcpyAsync(rec->x + (size_t)k * n, x, n * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream));
      SIE_CUDA(cudaMemcpyAsync(rec->r + (size_t)k * n, w, n * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream));
    }
    // V0 = r / beta (zero for finished right-hand sides)
    std::vector<zd> sc(R);
    for (int r = 0; r < R; ++r) sc[r] = active[r] ? zd(1.0 / rn[r], 0.0) : zd();
    SIE_CUDA(cudaMemcpyAsync(d_s, sc.data(), R * sizeof(zd), cudaMemcpyHostToDevice, c->stream));
    k_scale<<<gv, 256, 0, c->stream>>>(n, w, d_s, V);
    g.launch_check();
    std::fill(gvec.begin(), gvec.end(), cd(0.0));
    std::vector<zd> act(R);
    for (int r = 0; r < R; ++r) {
      gvec[(size_t)r * (m + 1)] = active[r] ? rn[r] : 0.0;
      if (active[r]) restarts[r]++;
      act[r] = zd(active[r] ? 1.0 : 0.0, 0.0);
    }
    SIE_CUDA(cudaMemcpyAsync(c->gm_act, act.data(), R * sizeof(zd), cudaMemcpyHostToDevice, c->stream));
    // z_j = M^-1 v_j and w = A z_j, as one captured graph per step (eagerly while the learned part is on)
    auto run_step = [&](int j) {
      zd *Vj = V + (size_t)j * vs, *Zj = Z + (size_t)j * vs;
      auto step = [&]() {
        if (precond >= 1) apply_ilu(c, Vj, Zj, R, prec);
        else SIE_CUDA(cudaMemcpyAsync(Zj, Vj, vs * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream));
        if (use_nn) nn_apply(c, Vj, Zj, R);
        apply_matvec(c, Zj, w, R, prec, 3);
      };
      if (use_nn) step();
      else SG.run(c, j, step);
    };
    zd *dh1 = d_h, *dh2 = d_h + (size_t)(m + 2) * R, *dnn = d_h + 2 * (size_t)(m + 2) * R;
    const zd *hp = (const zd *)c->gm_hpin;
    int jend = 0;
    run_step(0);
    for (int j = 0; j < m; ++j) {
      // classical Gram-Schmidt with a selective second pass, and the normalised
      // next vector, all on the device
      int *gate = (int *)c->gm_gate;
      double *npart = (double *)c->gm_npart;
      unsigned *cnt = (unsigned *)c->gm_cnt;
      // the previous step's Hessenberg copy (on the side stream) has read d_h
      if (j > 0) SIE_CUDA(cudaStreamWaitEvent(c->stream, c->gm_ev, 0));
      g.mdot(V, vs, j + 1, w, dh1);
      // first pass's update, |w'|^2 and the second-pass test
      SIE_CUDA(launch_chained(GS_CHAINED, k_orth_norm, gv, dim3(256), 0, c->stream, n, R, j + 1, (const zd *)V, vs,
                              (const zd *)dh1, w, (const int *)nullptr, npart, cnt, dnn, gate));
      g.launch_check();
      g.mdot(V, vs, j + 1, w, dh2, gate);
      SIE_CUDA(launch_chained(GS_CHAINED, k_orth_norm, gv, dim3(256), 0, c->stream, n, R, j + 1, (const zd *)V, vs,
                              (const zd *)dh2, w, (const int *)gate, npart, cnt, dnn, (int *)nullptr));
      g.launch_check();
      SIE_CUDA(launch_chained(GS_CHAINED, k_scale_norm, gv, dim3(256), 0, c->stream, n, (const zd *)w, (const zd *)dnn,
                              (const zd *)c->gm_act, V + (size_t)(j + 1) * vs));
      g.launch_check();
      // the Hessenberg column goes to the host on a side stream, so that the
      // next step does not wait for the copy
      SIE_CUDA(cudaEventRecord(c->gm_ev0, c->stream));
      SIE_CUDA(cudaStreamWaitEvent(c->gm_cs, c->gm_ev0, 0));
      SIE_CUDA(cudaMemcpyAsync(c->gm_hpin, d_h, 3 * (size_t)(m + 2) * R * sizeof(zd), cudaMemcpyDeviceToHost,
                               c->gm_cs));
      SIE_CUDA(cudaEventRecord(c->gm_ev, c->gm_cs));
      // the next step goes to the GPU before the host looks at the Hessenberg column:
      // if the cycle stops here, its result is simply not used
      if (j + 1 < m) run_step(j + 1);
      SIE_CUDA(cudaEventSynchronize(c->gm_ev));
      for (int r = 0; r < R; ++r) {
        cd *Hc = &H[((size_t)r * (m + 1)) * m];  // column-major per RHS: H[i + j (m+1)]
        for (int i = 0; i <= j; ++i) {
          const zd a1 = hp[(size_t)i * R + r], a2 = hp[(size_t)(m + 2) * R + (size_t)i * R + r];
          Hc[i + (size_t)j * (m + 1)] = cd(a1.re + a2.re, a1.im + a2.im);
        }
        Hc[j + 1 + (size_t)j * (m + 1)] = sqrt_nonneg(hp[2 * (size_t)(m + 2) * R + r].re);
      }
      // Givens rotations per RHS
      bool all_done = true;
      for (int r = 0; r < R; ++r) {
        cd *Hc = &H[((size_t)r * (m + 1)) * m];
        double *csr = &cs[(size_t)r * m];
        cd *snr = &sn[(size_t)r * m];
        cd *gr = &gvec[(size_t)r * (m + 1)];
        if (!active[r]) continue;
        for (int i = 0; i < j; ++i) {
          cd a = Hc[i + (size_t)j * (m + 1)], bb = Hc[i + 1 + (size_t)j * (m + 1)];
          Hc[i + (size_t)j * (m + 1)] = csr[i] * a + snr[i] * bb;
          Hc[i + 1 + (size_t)j * (m + 1)] = -std::conj(snr[i]) * a + csr[i] * bb;
        }
        cd a = Hc[j + (size_t)j * (m + 1)], bb = Hc[j + 1 + (size_t)j * (m + 1)];
        double cc;
        cd ss;
        if (std::abs(bb) == 0.0) { cc = 1.0; ss = 0.0; }
        else if (std::abs(a) == 0.0) { cc = 0.0; ss = 1.0; }
        else {
          double t = std::sqrt(std::norm(a) + std::norm(bb));
          cc = std::abs(a) / t;
          ss = (a / std::abs(a)) * std::conj(bb) / t;
        }
        csr[j] = cc;
        snr[j] = ss;
        Hc[j + (size_t)j * (m + 1)] = cc * a + ss * bb;
        Hc[j + 1 + (size_t)j * (m + 1)] = 0.0;
        gr[j + 1] = -std::conj(ss) * gr[j];
        gr[j] = cc * gr[j];
        iters[r]++;
        double est = std::abs(gr[j + 1]) / bn[r];
        if (!std::isfinite(est)) status = SIE_EBREAKDOWN;
        if (est > tol && iters[r] < max_iters) all_done = false;
      }
      total++;
      jend = j + 1;
      if (all_done || status != SIE_OK) break;
    }
    // y = H^-1 g per RHS, x += Z y
    std::vector<zd> y((size_t)jend * R);
    for (int r = 0; r < R; ++r) {
      cd *Hc = &H[((size_t)r * (m + 1)) * m];
      cd *gr = &gvec[(size_t)r * (m + 1)];
      std::vector<cd> yy(jend);
      for (int i = jend - 1; i >= 0; --i) {
        cd s = gr[i];
        for (int k = i + 1; k < jend; ++k) s -= Hc[i + (size_t)k * (m + 1)] * yy[k];
        yy[i] = active[r] && std::abs(Hc[i + (size_t)i * (m + 1)]) > 0 ? s / Hc[i + (size_t)i * (m + 1)] : 0.0;
      }
      for (int i = 0; i < jend; ++i) y[(size_t)i * R + r] = zd(yy[i].real(), yy[i].imag());
    }
    zd *d_y = d_s;  // reuse
    SIE_CUDA(cudaMemcpyAsync(d_y, y.data(), y.size() * sizeof(zd), cudaMemcpyHostToDevice, c->stream));
    k_xupd<<<gv, 256, 0, c->stream>>>(n, R, jend, Z, vs, d_y, x);
    g.launch_check();
    if (status != SIE_OK) break;
  }
  SIE_CUDA(cudaStreamSynchronize(c->stream));
  check_device_error(c);
  bool conv = true;
  for (int r = 0; r < R; ++r) {
    if (st) {
      st[r].iters = iters[r];
      st[r].restarts = restarts[r];
      st[r].rel_residual = relres[r];
      st[r].converged = relres[r] <= tol ? 1 : 0;
    }
    if (!(relres[r] <= tol)) conv = false;
  }
  (void)total;
  if (status != SIE_OK) return status;
  return conv ? SIE_OK : SIE_ENOTCONV;
}

// BiCGStab (method 1) and CGS (method 2), right-preconditioned, for R
// right-hand sides in lockstep on internal-order FP64 vectors; the inner
// operator and preconditioner in `prec`.  Scalars per right-hand side on the
// host.  When the recurrence residual of every active right-hand side is
// below tol, the true residual b - A x with the residual operator decides; a
// right-hand side that is not there restarts from its current x (iterative
// refinement).  Breakdown (a zero inner product) also restarts.
sie_status run_bicg_internal(sie_ctx *c, const zd *b, zd *x, int R, int max_iters, double tol, sie_prec prec,
                             sie_prec rprec, int precond, int method, sie_solve_stats *st) {
  const int n = 2 * c->ne;
  const size_t vs = (size_t)R * n;
  ensure_work(c, R);
  constexpr int NV = 9;  // r, r0, p, v, s|u, t|q, ph, sh|uh, w
  if (c->bi_R != R) {
    c->bi_buf = dev_alloc(c, NV * vs * sizeof(zd));
    c->bi_coef = dev_alloc(c, 4 * (size_t)R * sizeof(zd));
    c->bi_part = dev_alloc(c, (size_t)4 * R * ((n + 1023) / 1024) * sizeof(zd));
    c->bi_dot = dev_alloc(c, 4 * (size_t)R * sizeof(zd));
    c->bi_R = R;
  }
  zd *B = (zd *)c->bi_buf;
  zd *r = B, *r0 = B + vs, *p = B + 2 * vs, *v = B + 3 * vs, *s_ = B + 4 * vs, *t = B + 5 * vs, *ph = B + 6 * vs,
     *sh = B + 7 * vs, *w = B + 8 * vs;
  zd *cf = (zd *)c->bi_coef, *dd = (zd *)c->bi_dot;
  Gm g{c, n, R, std::max(1, (n + 1023) / 1024), (zd *)c->bi_part};
  dim3 gv((n + 255) / 256, R);
  auto precon = [&](const zd *in, zd *out) {
    if (precond >= 1) apply_ilu(c, in, out, R, prec);
    else SIE_CUDA(cudaMemcpyAsync(out, in, vs * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream));
  };
  // per right-hand-side dots <a[r], b[r]> -> host
  auto dots = [&](const zd *a, const zd *bb, std::vector<cd> &out) {
    g.mdot(a, 0, 1, bb, dd);
    std::vector<zd> h(R);
    SIE_CUDA(cudaMemcpyAsync(h.data(), dd, R * sizeof(zd), cudaMemcpyDeviceToHost, c->stream));
    SIE_CUDA(cudaStreamSynchronize(c->stream));
    out.resize(R);
    for (int q = 0; q < R; ++q) out[q] = cd(h[q].re, h[q].im);
  };
  auto coef = [&](int slot, const std::vector<cd> &vals) {
    std::vector<zd> h(R);
    for (int q = 0; q < R; ++q) h[q] = zd(vals[q].real(), vals[q].imag());
    SIE_CUDA(cudaMemcpyAsync(cf + (size_t)slot * R, h.data(), R * sizeof(zd), cudaMemcpyHostToDevice, c->stream));
    return cf + (size_t)slot * R;
  };
  auto axpy = [&](const zd *a, const std::vector<cd> &k, const zd *bb, zd *out, int slot) {
    k_axpy_r<<<gv, 256, 0, c->stream>>>(n, a, coef(slot, k), bb, out);
    g.launch_check();
  };
  std::vector<cd> bn2, rn2;
  dots(b, b, bn2);
  std::vector<double> bn(R);
  for (int q = 0; q < R; ++q) bn[q] = sqrt_nonneg(bn2[q].real());
  std::vector<int> iters(R, 0), restarts(R, 0), active(R, 1);
  std::vector<double> relres(R, 0.0);
  sie_status status = SIE_OK;
  const std::vector<cd> one(R, cd(1.0)), mone(R, cd(-1.0));
  auto relnorm = [&](const std::vector<cd> &nn, int q) {
    return bn[q] > 0 ? sqrt_nonneg(nn[q].real()) / bn[q] : (std::isnan(bn[q]) ? bn[q] : 0.0);
  };
  std::vector<cd> xn2;
  dots(x, x, xn2);
  bool x_zero = true;
  for (int q = 0; q < R; ++q) x_zero = x_zero && xn2[q].real() == 0.0;
  int stalls = 0;  // restarts in a row without a single step (repeated breakdown)
  for (bool first_cycle = true;; first_cycle = false) {
    // true residual with the residual operator rprec (r = b for a zero initial guess)
    if (first_cycle && x_zero) {
      SIE_CUDA(cudaMemcpyAsync(r, b, vs * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      apply_matvec(c, x, w, R, rprec, 3);
      axpy(b, mone, w, r, 0);
    }
    dots(r, r, rn2);
    check_device_error(c);
    bool any = false;
    for (int q = 0; q < R; ++q) {
      relres[q] = relnorm(rn2, q);
      if (!std::isfinite(relres[q])) status = SIE_EBREAKDOWN;
      active[q] = relres[q] > tol && iters[q] < max_iters && std::isfinite(relres[q]);
      if (active[q]) {
        any = true;
        restarts[q]++;
      }
    }
    if (!any || status != SIE_OK) break;
    SIE_CUDA(cudaMemcpyAsync(r0, r, vs * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream));
    SIE_CUDA(cudaMemsetAsync(p, 0, vs * sizeof(zd), c->stream));
    SIE_CUDA(cudaMemsetAsync(v, 0, vs * sizeof(zd), c->stream));  // CGS: q
    std::vector<cd> rho_old(R, cd(1.0)), alpha(R, cd(1.0)), omega(R, cd(1.0)), rho;
    bool first = true, breakdown = false;
    int steps = 0;
    for (;;) {
      dots(r0, r, rho);
      std::vector<cd> k1(R, 0.0), k2(R, 0.0), k3(R, 0.0);
      for (int q = 0; q < R; ++q)
        if (active[q] && (rho[q] == 0.0 || !std::isfinite(std::abs(rho[q])))) breakdown = true;
      if (breakdown) break;
      if (method == 1) {
        // p = r + beta (p - omega v)
        for (int q = 0; q < R; ++q)
          if (active[q]) {
            const cd beta = first ? cd(0.0) : (rho[q] / rho_old[q]) * (alpha[q] / omega[q]);
            k1[q] = beta;
            k2[q] = -omega[q];
          }
        k_axpy2_r<<<gv, 256, 0, c->stream>>>(n, r, coef(0, k1), p, coef(1, k2), v, p);
        g.launch_check();
        precon(p, ph);
        apply_matvec(c, ph, v, R, prec, 3);
        std::vector<cd> rv;
        dots(r0, v, rv);
        for (int q = 0; q < R; ++q) {
          if (!active[q]) continue;
          if (rv[q] == 0.0) breakdown = true;
          alpha[q] = rho[q] / rv[q];
          k1[q] = -alpha[q];
        }
        if (breakdown) break;
        axpy(r, k1, v, s_, 2);  // s = r - alpha v (r for finished right-hand sides)
        precon(s_, sh);
        apply_matvec(c, sh, t, R, prec, 3);
        std::vector<cd> ts, tt;
        dots(t, s_, ts);
        dots(t, t, tt);
        for (int q = 0; q < R; ++q) {
          k1[q] = k2[q] = 0.0;
          if (!active[q]) continue;
          omega[q] = tt[q].real() > 0 ? ts[q] / tt[q] : cd(0.0);  // t = 0 only when s = 0
          k1[q] = alpha[q];
          k2[q] = omega[q] / (alpha[q] == 0.0 ? cd(1.0) : alpha[q]);
        }
        // x += alpha (ph + (omega / alpha) sh);  r = s - omega t
        k_axpy2_r<<<gv, 256, 0, c->stream>>>(n, x, coef(0, k1), ph, coef(1, k2), sh, x);
        g.launch_check();
        for (int q = 0; q < R; ++q) k3[q] = active[q] ? -omega[q] : cd(0.0);
        axpy(s_, k3, t, r, 2);
      } else {
        // u = r + beta q;  p = u + beta (q + beta p)
        zd *u = s_, *qv = v;
        for (int q = 0; q < R; ++q)
          if (active[q]) k1[q] = first ? cd(0.0) : rho[q] / rho_old[q];
        axpy(r, k1, qv, u, 0);
        k_axpy2_r<<<gv, 256, 0, c->stream>>>(n, u, coef(1, k1), qv, coef(2, k1), p, p);
        g.launch_check();
        precon(p, ph);
        apply_matvec(c, ph, t, R, prec, 3);  // t = A M^-1 p
        std::vector<cd> rv;
        dots(r0, t, rv);
        for (int q = 0; q < R; ++q) {
          k1[q] = 0.0;
          if (!active[q]) continue;
          if (rv[q] == 0.0) breakdown = true;
          alpha[q] = rho[q] / rv[q];
          k1[q] = -alpha[q];
        }
        if (breakdown) break;
        axpy(u, k1, t, qv, 0);              // q = u - alpha t
        axpy(u, one, qv, w, 1);             // w = u + q
        precon(w, sh);                       // uh = M^-1 (u + q)
        for (int q = 0; q < R; ++q) k2[q] = -k1[q];
        axpy(x, k2, sh, x, 2);               // x += alpha uh
        apply_matvec(c, sh, t, R, prec, 3);
        axpy(r, k1, t, r, 3);                // r -= alpha A uh
      }
      first = false;
      ++steps;
      rho_old = rho;
      dots(r, r, rn2);
      bool all_done = true;
      for (int q = 0; q < R; ++q) {
        if (!active[q]) continue;
        iters[q]++;
        const double e = relnorm(rn2, q);
        if (!std::isfinite(e)) {
          status = SIE_EBREAKDOWN;
          break;
        }
        if (e <= tol || iters[q] >= max_iters) active[q] = 0;  // frozen: coefficients 0 from now on
        else all_done = false;
      }
      if (all_done || status != SIE_OK) break;
    }
    if (status != SIE_OK) break;
    stalls = steps == 0 ? stalls + 1 : 0;
    if (breakdown && stalls >= 2) {
      status = SIE_EBREAKDOWN;
      break;
    }
  }
  SIE_CUDA(cudaStreamSynchronize(c->stream));
  check_device_error(c);
  bool conv = true;
  for (int q = 0; q < R; ++q) {
    if (st) {
      st[q].iters = iters[q];
      st[q].restarts = restarts[q];
      st[q].rel_residual = relres[q];
      st[q].converged = relres[q] <= tol ? 1 : 0;
    }
    if (!(relres[q] <= tol)) conv = false;
  }
  if (status != SIE_OK) return status;
  return conv ? SIE_OK : SIE_ENOTCONV;
}

// Operator of the true residual.  The plain form keeps every step in FP64.
// The mixed form uses the FP64 near field with the FP32 far field, whose
// rounding leaves the residual operator within a few 1e-6 (relative) of the
// FP64 operator: it decides convergence only for tolerances well above that
// floor, the whole FP64 operator below it (or on request).
sie_prec residual_prec(sie_prec prec, double tol, bool far_fp64) {
  constexpr double kNear64MinTol = 5e-5;
  return prec == SIE_PREC_MIXED && !far_fp64 && tol >= kNear64MinTol ? SIE_PREC_NEAR64 : SIE_PREC_FP64;
}

sie_status run_gmres(sie_ctx *c, const zd *b_user, zd *x_user, int R, const sie_solve_opts *o, sie_solve_stats *st) {
  const size_t vs = (size_t)R * 2 * c->ne;
  if (c->gw_R != R) {
    c->gm_b = dev_alloc(c, vs * sizeof(zd));
    c->gm_x = dev_alloc(c, vs * sizeof(zd));
    c->gw_R = R;
  }
  zd *b = (zd *)c->gm_b, *x = (zd *)c->gm_x;
  op_permute_in(c, b_user, b, R);
  op_permute_in(c, x_user, x, R);
  sie_prec prec = o->prec == 1 ? SIE_PREC_MIXED : SIE_PREC_FP64;
  const sie_prec rprec = residual_prec(prec, o->tol, o->residual_far_fp64 != 0);
  struct Eager {  // eager steps for this call only, also when it throws
    sie_ctx *c;
    ~Eager() { c->graphs_off = false; }
  } eager{c};
  c->graphs_off = o->no_graphs != 0;
  sie_status rc = o->method == 0
                      ? run_gmres_internal(c, b, x, R, o->restart, o->max_iters, o->tol, prec, rprec, o->precond,
                                           nullptr, st)
                      : run_bicg_internal(c, b, x, R, o->max_iters, o->tol, prec, rprec, o->precond, o->method, st);
  op_permute_out(c, x, x_user, R);
  SIE_CUDA(cudaStreamSynchronize(c->stream));
  return rc;
}

// out = a - b
void op_sub(sie_ctx *c, const zd *a, const zd *b, zd *out, int64_t n) {
  k_sub<<<std::max(1, (int)std::min<int64_t>(152 * 16, (n + 255) / 256)), 256, 0, c->stream>>>(n, a, b, out);
  SIE_CHECK_LAUNCH();
  c->launches++;
}
