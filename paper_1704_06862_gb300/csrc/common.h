// Internal declarations of the GB300 JMCFIE/MLFMM library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <cstdio>
#include <string>
#include <array>
#include <vector>

#include "sie.h"

#define SIE_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------------ launch chaining
// Programmatic dependent launch: a kernel launched with chained = true may
// start while its predecessor on the stream drains.  It reads only static
// data (tables, factors, pointers) before pdl_wait(), which returns once the
// predecessor has completed and its writes are visible; pdl_release(), issued
// after the wait, lets the next kernel launch, so a kernel never overlaps the
// one two back.  Without the launch attribute both are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(bool chained, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                           cudaStream_t st, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = chained ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// Cooperative launch: every CTA of the grid is resident at once (the driver
// refuses the launch otherwise), which a grid barrier inside the kernel needs.
template <typename... KArgs, typename... Args>
cudaError_t launch_cooperative(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// ------------------------------------------------------------------ complex
template <typename T>
struct cx {
  T re, im;
  SIE_HD cx() : re(0), im(0) {}
  SIE_HD cx(T r, T i = 0) : re(r), im(i) {}
  template <typename U>
  SIE_HD explicit cx(const cx<U> &o) : re((T)o.re), im((T)o.im) {}
};
template <typename T> SIE_HD cx<T> operator+(cx<T> a, cx<T> b) { return cx<T>(a.re + b.re, a.im + b.im); }
template <typename T> SIE_HD cx<T> operator-(cx<T> a, cx<T> b) { return cx<T>(a.re - b.re, a.im - b.im); }
template <typename T> SIE_HD cx<T> operator-(cx<T> a) { return cx<T>(-a.re, -a.im); }
template <typename T> SIE_HD cx<T> operator*(cx<T> a, cx<T> b) {
  return cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> SIE_HD cx<T> operator*(T s, cx<T> a) { return cx<T>(s * a.re, s * a.im); }
template <typename T> SIE_HD cx<T> operator*(cx<T> a, T s) { return cx<T>(s * a.re, s * a.im); }
template <typename T> SIE_HD cx<T> &operator+=(cx<T> &a, cx<T> b) { a.re += b.re; a.im += b.im; return a; }
template <typename T> SIE_HD cx<T> &operator-=(cx<T> &a, cx<T> b) { a.re -= b.re; a.im -= b.im; return a; }
template <typename T> SIE_HD cx<T> conj(cx<T> a) { return cx<T>(a.re, -a.im); }
template <typename T> SIE_HD cx<T> cfma(cx<T> a, cx<T> b, cx<T> c) {  // a*b + c
  return cx<T>(fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im)));
}
typedef cx<double> zd;
typedef cx<float> zf;

// ------------------------------------------------------------------ errors
struct SieError {
  sie_status code;
  std::string msg;
};
#define SIE_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw SieError{SIE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};         \
  } while (0)
#define SIE_CHECK_LAUNCH() SIE_CUDA(cudaGetLastError())
#define SIE_REQUIRE(cond, code, msg)       \
  do {                                     \
    if (!(cond)) throw SieError{code, msg}; \
  } while (0)

// ------------------------------------------------------------------ device buffers
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

// ------------------------------------------------------------------ one octree level of one medium
struct LevelHost {
  int lev = 0;       // level number (0 = root)
  double a = 0;      // box edge
  int L = 0, K = 0;  // truncation and number of directions (L+1)(2L+2)
  int nbox = 0;
  std::vector<int> ijk;       // [nbox][3]
  std::vector<int> parent;    // index in level lev-1
  std::vector<int> oct;       // octant of the box in its parent (bit0 x, bit1 y, bit2 z)
  std::vector<int> ch_ptr, ch_idx;        // children CSR (level lev+1)
  std::vector<int> il_ptr, il_src, il_slot;  // interaction list CSR, translator slot
  std::vector<int> slot_code;             // offset code per translator slot
  // device tables
  double *d_dirs = nullptr;     // [K][9]: khat, theta_hat, phi_hat
  void *d_T64 = nullptr, *d_T32 = nullptr;       // translators [nslot][K], weights and constants folded
  void *d_tp64 = nullptr, *d_tp32 = nullptr;     // [K][6]: theta_hat, phi_hat
  // separable interpolation to this level from lev+1 (real): Phi [Np][Nc], Theta+- [L+1][Lc+1]
  void *d_Phi64 = nullptr, *d_Phi32 = nullptr, *d_Thp64 = nullptr, *d_Thp32 = nullptr;
  void *d_Thm64 = nullptr, *d_Thm32 = nullptr;
  void *d_up64 = nullptr, *d_up32 = nullptr;     // [8][K] shift, child -> this (parent) level
  void *d_dn64 = nullptr, *d_dn32 = nullptr;     // [8][K] shift, this level -> child
  int *d_il_ptr = nullptr, *d_il_src = nullptr, *d_il_slot = nullptr;
  // sibling groups (the children of one box of the level above) for the M2L:
  // per group up to 8 member boxes and the union of their interaction lists,
  // one entry per source: (source box, member mask, translator slot per member)
  int ngroups = 0, max_group_entries = 0;
  int *d_grp_ptr = nullptr, *d_grp_box = nullptr, *d_grp_ent = nullptr;
  int *d_ch_ptr = nullptr, *d_ch_idx = nullptr, *d_oct = nullptr, *d_parent = nullptr;
  // work buffers (capacity nrhs_cap): S and I [nbox][2][2][K][R]
  void *d_S = nullptr, *d_I = nullptr;
};

struct RegionHost {
  int id = 0;
  std::complex<double> k, eta;  // wavenumber, relative impedance eta_l / eta_0
  int nb = 0;                   // bases of this medium
  std::vector<int> basis_p;     // internal edge index
  std::vector<int> basis_sign;  // s_l
  std::vector<int> box_start;   // leaf boxes: [nleaf+1] ranges into the basis list
  int max_leaf = 0;             // most bases in one leaf box
  std::vector<LevelHost> lev;   // index = level number; levels top..leaf carry tables
  // coarsest level whose interaction lists are not empty (2 unless the medium's
  // bases sit in mutually adjacent boxes there): coarser levels translate
  // nothing, so they are neither aggregated into nor given directions
  int top = 2;
  int *d_basis_p = nullptr, *d_basis_sign = nullptr, *d_box_start = nullptr, *d_basis_box = nullptr;
  // per basis of the medium: its two triangles in this medium and the sign of
  // each triangle's piece in the radiation pattern (1, 1 for an ordinary edge,
  // whose medium sign is basis_sign; s_l(T) for a junction edge, basis_sign 1)
  std::vector<int> ptri;
  std::vector<double> psg;
  int *d_ptri = nullptr;
  double *d_psg = nullptr;
  int rpart_off = 0;            // first row of this medium in the concatenated receive outputs
  double *d_box_centre = nullptr;  // leaf box centres [nleaf][3]
  void *d_V64 = nullptr, *d_V32 = nullptr;    // radiation patterns [nb][2][Kleaf]
  void *d_P64 = nullptr, *d_P32 = nullptr;  // combined receive patterns [nb][2][Kleaf] (k_receive_fold)
  // the radiation patterns as the pre-split A operand of the tensor-core
  // aggregation (tensor.cu: per box, chunks in the shared-memory byte layout)
  void *d_agg_op = nullptr;
  int64_t *d_agg_off = nullptr;   // [nleaf+1] byte offsets of the boxes
  size_t agg_op_bytes = 0;
  // the combined receive patterns as the pre-split A operand of the tensor-core receive
  void *d_rec_op = nullptr;
  int64_t *d_rec_off = nullptr;
  size_t rec_op_bytes = 0;
  int *d_pairs = nullptr;       // near triangle pairs (p, q, singular) for the fill
  int64_t npairs = 0;
};

struct IluHost {
  bool ready = false;
  int nboxes = 0;
  std::vector<int> colour_ptr;     // boxes grouped by colour: [9]
  int *d_box_start = nullptr;      // [nbox+1] internal edge ranges
  int *d_box_list = nullptr;       // boxes in colour order
  int *d_lo_ptr = nullptr, *d_lo_col = nullptr, *d_up_ptr = nullptr, *d_up_col = nullptr;
  // per row, [9] starts of each column colour's blocks within its off-box range (the 9th = end)
  int *d_lo_cptr = nullptr, *d_up_cptr = nullptr;
  // single-RHS sweep steps (forward colours 0..7, backward 6..0): pieces of the
  // boxes' off-box work, 5 ints each (box, v0, v1, index in box, pieces of box);
  // step s uses pieces [piece_ptr[s], piece_ptr[s+1])
  std::vector<int> piece_ptr;
  int *d_pieces = nullptr;
  int *d_piece_count = nullptr;     // per box arrival counter (self-resetting)
  void *d_piece_scratch = nullptr;  // per piece row partials [piece][2 max_box] complex (FP64 size)
  void *d_lo64 = nullptr, *d_lo32 = nullptr, *d_up64 = nullptr, *d_up32 = nullptr;  // off-box blocks [.][4]
  // in-box inverses packed by rows, per box: strictly lower part of L_bb^{-1}
  // (its diagonal blocks are identities; row i holds blocks j < i) and the
  // upper part, diagonal included, of U_bb^{-1} (row i holds blocks j >= i)
  int64_t *d_tl_off = nullptr, *d_tu_off = nullptr;  // per box offsets, in blocks
  void *d_tl64 = nullptr, *d_tl32 = nullptr, *d_tu64 = nullptr, *d_tu32 = nullptr;
  int max_box = 0;
  int64_t nblk_off = 0, nblk_inv = 0;  // off-box factor blocks (L and U); in-box inverse blocks
  unsigned *d_bar = nullptr;  // grid-barrier arrival count of the persistent apply (cleared before each launch)
};

// most right-hand sides per product whose leaf receives run concurrently (one
// output block per medium, then a combine in medium order); larger blocks
// receive one medium after another directly into y
constexpr int RPART_MAX_RHS = 8;

struct sie_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  int64_t launches = 0;
  int64_t dev_bytes = 0;
  std::vector<DBuf> bufs;

  // mesh
  bool have_mesh = false, have_tree = false, have_fill = false;
  double freq = 0, k0 = 0;
  int nv = 0, nt = 0, nr = 0, ne = 0;
  std::vector<double> verts;            // [nv][3]
  std::vector<int> tris, tri_reg;       // [nt][3], [nt][2]
  std::vector<double> media;            // [nr][4]
  std::vector<double> area, normal, centroid, hmax;
  std::vector<int> edge_v, tp, tm, vp, vm;  // user edge numbering
  std::vector<double> elen;
  std::vector<int> tri_edge, tri_free;  // [nt][3] user edge index / free vertex
  std::vector<double> tri_sign;         // [nt][3] coefficient of the edge's function on the triangle:
                                        // +1 on T+, -1 on T-; a_T at a junction edge
  // per edge: the media it lies in, each with its two triangles (region, T1, T2);
  // two entries for an ordinary edge, one per touching region at a junction
  std::vector<int> emed_ptr;
  std::vector<std::array<int, 3>> emed;
  std::vector<char> ejunc;              // per edge: 1 at a junction
  int njunc = 0;                        // junction edges
  std::vector<std::complex<double>> kreg, etareg;

  // tree and ordering
  int levels = 0;
  double digits = 3;
  double origin[3] = {0, 0, 0}, D = 0, hleaf = 0;
  std::vector<int> perm, inv;           // perm[p] = user edge; inv[user] = p
  std::vector<int> eijk;                // [ne][3] leaf box of each user edge
  std::vector<int> leaf_start;          // global leaf boxes (internal order): edge ranges
  std::vector<int> leaf_ijk;
  std::vector<int> row_ptr, col;        // near pattern (internal indices), sorted rows
  std::vector<RegionHost> reg;
  IluHost ilu;

  // device geometry
  double *d_tri = nullptr;       // per triangle: 3 verts (9), normal (3), area (1), free verts (9) = 22 doubles
  int *d_tri_e = nullptr;        // per triangle: 3 internal edge ids (-1 none)
  double *d_tri_sg = nullptr;    // per triangle: 3 signs * len/(2A)
  int *d_tri_reg = nullptr;      // [nt][2]
  bool graphs_off = false;       // Krylov steps launched eagerly (sie_solve_opts.no_graphs)
  int form = 0;                  // sie_fill_opts.formulation
  std::vector<std::complex<double>> rowscale;  // ICTF: per basis (J-row, M-row) weights, internal order
  void *d_rowscale = nullptr;                  // the same on the device [ne][2]
  int *d_tri0 = nullptr;         // triangles bounding the host medium (region 0)
  int ntri0 = 0;
  void *d_ff = nullptr;          // far-field work: point positions, point currents, partial sums
  size_t ff_bytes = 0;
  int *d_row_ptr = nullptr, *d_col = nullptr;
  void *d_near64 = nullptr, *d_near32 = nullptr;  // [nnzb][4] blocks
  int *d_perm = nullptr, *d_inv = nullptr;
  int *d_edge_tris = nullptr;    // per internal edge: its two triangles in medium 0 (-1: not on medium 0)
  double *d_quad = nullptr;      // outer singular rule (b0,b1,b2,w) * nq
  int nq_sing = 16;

  // work buffers
  int64_t nrhs_cap = 0;
  void *d_xi = nullptr, *d_yi = nullptr;          // internal-order FP64 vectors [R][ne][2]
  void *d_xf = nullptr, *d_yf = nullptr;          // FP32 copies
  void *d_scratch = nullptr;                      // upward-pass child contributions, one slice per medium
  size_t scratch_region = 0;                      // bytes of one medium's slice
  // concurrent receives (blocks of up to RPART_MAX_RHS right-hand sides): each
  // medium writes its rows [r][rpart_nb][2] here, a combine kernel adds them
  // into y in medium order; d_rmap [ne][2]: a basis's rows (lower medium first)
  void *d_iluT = nullptr;        // block ILU(0): interleaved source and result, [2][n][iluT_R] (FP64 capacity)
  int iluT_R = 0;
  void *d_rpart = nullptr;
  int rpart_cap = 0, rpart_nb = 0;
  int *d_rmap = nullptr;
  std::vector<cudaStream_t> rstream;              // one stream per medium for the far-field passes
  std::vector<cudaEvent_t> ev_join;               // end of each medium's passes
  cudaEvent_t ev_fork = nullptr;                  // start of the far field on the context stream
  void *d_stage = nullptr;                        // small host-to-device staging area
  size_t stage_bytes = 0;
  // Krylov storage of the last solve shape (restart m, nrhs R)
  int gm_m = 0, gm_R = 0, gw_R = 0;
  int bi_R = 0;  // BiCGStab / CGS work vectors, per block size
  void *bi_buf = nullptr, *bi_coef = nullptr, *bi_part = nullptr, *bi_dot = nullptr;
  int64_t work_gen = 0;     // bumped whenever work buffers are (re)allocated
  void *graphs = nullptr;   // captured per-step operator graphs (solve.cu)
  void *nn = nullptr;  // learned-preconditioner state (nn.cu)
  void *gm_V = nullptr, *gm_Z = nullptr, *gm_b = nullptr, *gm_x = nullptr, *gm_w = nullptr;
  void *gm_h = nullptr, *gm_s = nullptr, *gm_part = nullptr, *gm_act = nullptr, *gm_gate = nullptr;
  void *gm_hpin = nullptr;        // pinned host mirror of gm_h (one copy per Krylov step)
  cudaEvent_t gm_ev = nullptr;    // marks that copy (made on gm_cs)
  cudaStream_t gm_cs = nullptr;   // side stream of the copy
  cudaEvent_t gm_ev0 = nullptr;   // the step's Gram-Schmidt done (gm_cs waits on it)
  void *gm_npart = nullptr;       // per-CTA partial norms of the fused update
  void *gm_cnt = nullptr;         // completion counter of the fused update (self-resetting)
  // bounded device-side waits: polls before a wait gives up, and the flag a
  // kernel sets when one did (read and cleared by sie_device_status and the solvers)
  int wait_limit = 1 << 21;
  int *d_err = nullptr;
  int ilu_schedule = 1;           // single-RHS ILU apply: 0 persistent cooperative launch, 1 one launch per step
  // tensor-core leaf aggregation (FP32 operator, blocks of right-hand sides):
  // used from agg_tc_min_rhs right-hand sides on (0: never), agg_tc_rb per pass (0: by block size)
  int agg_tc_min_rhs = 16, agg_tc_rb = 0;
  // tile shapes of the block-RHS kernels (0 or -1: the built-in rule; set by
  // sie_set_param or chosen by sie_autotune): right-hand sides per block load
  // of the near-field product and the ILU sweeps, per pass of the leaf
  // receive; M2L form (0 per target box, 1 by sibling groups, 2 by sibling
  // groups split over warps)
  int tune_near_rb = 0, tune_ilu_rb = 0, tune_rec_rb = 0, tune_m2l = -1;
  // tensor-core leaf receive: right-hand sides per pass (0: the SIMT receive,
  // -1: from 16 right-hand sides on, by the block size)
  int rec_tc_rb = -1;
  // learned-preconditioner layers X W^T on the tensor cores (1) or the SIMT tiles (0)
  int nn_tc = 1;
  // interpolation and anterpolation CTAs per (box, right-hand side): -1 (one per
  // source for one right-hand side on levels of fewer than 2048 boxes, else
  // one), 0 one for both sources J, M, 1 one per source
  int tune_interp_split = -1;
};

// ------------------------------------------------------------------ host helpers (host.cpp)
void *dev_alloc(sie_ctx *c, size_t bytes);
template <typename T>
T *dev_upload(sie_ctx *c, const std::vector<T> &v) {
  if (v.empty()) return nullptr;
  T *p = (T *)dev_alloc(c, v.size() * sizeof(T));
  SIE_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}
void ensure_work(sie_ctx *c, int64_t nrhs);
void *stage(sie_ctx *c, size_t bytes);
// throws SIE_ETIMEOUT if a device-side wait gave up since the last check
// (synchronises the context stream; clears the record)
void check_device_error(sie_ctx *c);
void region_streams(sie_ctx *c);  // creates the per-medium streams and events once
// weights (aTJ, aNJ, aTM, aNM) of medium l for the context's formulation
void form_weights(const sie_ctx *c, int l, std::complex<double> w[4]);
// ICTF: y[r][p][j] *= rowscale[p][j] (no-op for the other formulations)
void op_rowscale(sie_ctx *c, zd *y, int nrhs);

// ------------------------------------------------------------------ launchers (fill.cu)
void launch_near_fill(sie_ctx *c, int region);
void launch_identity(sie_ctx *c);
void launch_patterns(sie_ctx *c, int region);
void launch_rhs(sie_ctx *c, const double *inc_dev, int nrhs, zd *b_internal);
void launch_farfield(sie_ctx *c, const zd *x_internal, int nrhs, const double *obs_dev, int nobs, double *out_dev,
                     sie_prec prec);
void launch_to_f32(sie_ctx *c, const double *src, float *dst, int64_t n);

// ------------------------------------------------------------------ launchers (operator.cu)
template <typename T>
void op_near(sie_ctx *c, const cx<T> *x, cx<T> *y, int nrhs, bool accumulate);
// forked: far_fork already recorded; TY: type of the product y the receives add into
template <typename T, typename TY = T>
void op_far(sie_ctx *c, const cx<T> *x, cx<TY> *y, int nrhs, bool forked = false);
void far_fork(sie_ctx *c);
template <typename T>
void op_ilu(sie_ctx *c, const cx<T> *r, cx<T> *z, int nrhs);
// tensor-core leaf aggregation (tensor.cu): right-hand sides per pass for a
// block of nrhs (0: the SIMT kernel is used), and the launch for one medium
int agg_tc_block(const sie_ctx *c, int nrhs);
int rec_tc_block(const sie_ctx *c, int nrhs);
bool op_aggregate_tc(sie_ctx *c, int rb, int K, int nbox, int max_leaf, int nrhs, const int *box_start,
                     const int64_t *box_off, const int *basis_p, const int *sign, const unsigned char *Aop,
                     const zf *x, zf *S, cudaStream_t st);
void build_agg_operand(sie_ctx *c, RegionHost &R, int K);  // at setup, after the FP32 patterns
// tensor-core leaf receive (tensor.cu): adds the medium's far field into the FP32 product y
// one dense layer act(X W^T + bias) of the learned preconditioner on the
// tensor cores (BF16 X [M][K], W [N][K]); false when the shape is not covered
bool nn_dense_tc(sie_ctx *c, int M, int N, int K, const void *X, const void *W, const float *bias, int relu,
                 float *Cf, void *Cb);
bool op_receive_tc(sie_ctx *c, int rb, int K, int nbox, int nrhs, const int *box_start, const int64_t *box_off,
                   const int *basis_p, const unsigned char *Aop, const zf *I, zf eta, zf ieta, zf cJ, zf cM, zf *y,
                   cudaStream_t st);
void build_rec_operand(sie_ctx *c, RegionHost &R, int K);  // at setup, after the FP32 receive patterns
void op_permute_in(sie_ctx *c, const zd *user, zd *internal, int nrhs);    // user -> internal
void op_permute_out(sie_ctx *c, const zd *internal, zd *user, int nrhs);   // internal -> user
void op_d2f(sie_ctx *c, const zd *a, zf *b, int64_t n);
void op_f2d(sie_ctx *c, const zf *a, zd *b, int64_t n);

// operator on internal-order FP64 vectors, in the requested arithmetic
void apply_matvec(sie_ctx *c, const zd *x, zd *y, int nrhs, sie_prec prec, int parts);
void apply_ilu(sie_ctx *c, const zd *r, zd *z, int nrhs, sie_prec prec);

// ------------------------------------------------------------------ solver (solve.cu)
sie_status run_gmres(sie_ctx *c, const zd *b_user, zd *x_user, int nrhs, const sie_solve_opts *o,
                     sie_solve_stats *st);
struct Recorder {  // training pairs taken at the restarts of one solve
  zd *x, *r;       // [cap][2 ne] internal order
  int cap;
  int *count;
};
// operator of the true residual for inner precision prec and tolerance tol
sie_prec residual_prec(sie_prec prec, double tol, bool far_fp64);
// prec: inner operator and preconditioner; rprec: operator of the true residual
sie_status run_gmres_internal(sie_ctx *c, const zd *b, zd *x, int R, int m, int max_iters, double tol,
                              sie_prec prec, sie_prec rprec, int precond, Recorder *rec, sie_solve_stats *st);
void op_sub(sie_ctx *c, const zd *a, const zd *b, zd *out, int64_t n);
void graphs_free(sie_ctx *c);
// Krylov step graphs: -1 none captured yet, 0 capture failed (steps run eagerly), 1 in use
int graphs_state(const sie_ctx *c);

// ------------------------------------------------------------------ learned preconditioner (nn.cu)
bool nn_ready(sie_ctx *c);
bool nn_trained(sie_ctx *c);
void nn_apply(sie_ctx *c, const zd *v, zd *z, int nrhs);
void nn_free(sie_ctx *c);
