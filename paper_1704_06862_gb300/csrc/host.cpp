// Host side of the library: mesh topology (RWG, Eq. 22), octree, near-field
// pattern and preconditioner ordering, MLFMM tables, ILU(0) factorisation,
// and the extern "C" entry points declared in sie.h.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>
#include <unordered_map>

#include "common.h"

typedef std::complex<double> cd;
static const double PI = 3.14159265358979323846;

// ------------------------------------------------------------------ allocation
void *dev_alloc(sie_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) throw SieError{SIE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  c->bufs.push_back({p, bytes});
  c->dev_bytes += (int64_t)bytes;
  return p;
}

void form_weights(const sie_ctx *c, int l, std::complex<double> w[4]) {
  const std::complex<double> e = c->etareg[l];
  switch (c->form) {
    case 1: w[0] = 1.0; w[1] = 0.0; w[2] = 1.0; w[3] = 0.0; break;        // CTF
    case 2: w[0] = 0.0; w[1] = 1.0; w[2] = 0.0; w[3] = 1.0; break;        // CNF
    case 3:                                                              // PMCHWT
    case 4: w[0] = e; w[1] = 0.0; w[2] = 1.0 / e; w[3] = 0.0; break;     // ICTF: PMCHWT rows, scaled per interface
    default: w[0] = w[1] = w[2] = w[3] = 1.0;                            // JMCFIE
  }
}

void region_streams(sie_ctx *c) {
  if (c->rstream.size() == c->reg.size() && c->ev_fork) return;
  if (!c->ev_fork) SIE_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  while (c->rstream.size() < c->reg.size()) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    SIE_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    SIE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->rstream.push_back(s);
    c->ev_join.push_back(e);
  }
}

void *stage(sie_ctx *c, size_t bytes) {
  if (bytes > c->stage_bytes) {
    c->d_stage = dev_alloc(c, std::max(bytes, (size_t)4096));
    c->stage_bytes = std::max(bytes, (size_t)4096);
  }
  return c->d_stage;
}

void check_device_error(sie_ctx *c) {
  if (!c->d_err) return;
  int e = 0;
  SIE_CUDA(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SIE_CUDA(cudaStreamSynchronize(c->stream));
  if (e) {
    // a launch that gave up may have left a box's piece count part-way
    if (c->ilu.d_piece_count)
      SIE_CUDA(cudaMemsetAsync(c->ilu.d_piece_count, 0, (size_t)c->ilu.nboxes * sizeof(int), c->stream));
    SIE_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    SIE_CUDA(cudaStreamSynchronize(c->stream));
    throw SieError{SIE_ETIMEOUT, "a bounded device-side wait gave up (grid barrier of the ILU(0) apply)"};
  }
}

void ensure_work(sie_ctx *c, int64_t nrhs) {
  if (nrhs <= c->nrhs_cap) return;
  size_t n = (size_t)nrhs * c->ne * 2;
  c->d_xi = dev_alloc(c, n * sizeof(zd));
  c->d_yi = dev_alloc(c, n * sizeof(zd));
  c->d_xf = dev_alloc(c, n * sizeof(zf));
  c->d_yf = dev_alloc(c, n * sizeof(zf));
  size_t scratch = 0;
  for (auto &R : c->reg) {
    for (int l = R.top; l < (int)R.lev.size(); ++l) {
      LevelHost &L = R.lev[l];
      size_t sz = (size_t)L.nbox * 4 * L.K * nrhs * sizeof(zd);
      L.d_S = dev_alloc(c, sz);
      L.d_I = dev_alloc(c, sz);
      if (l > R.top)  // children's interpolated patterns in the parent sampling
        scratch = std::max(scratch, (size_t)L.nbox * 4 * R.lev[l - 1].K * nrhs * sizeof(zd));
    }
  }
  c->scratch_region = (scratch + 255) / 256 * 256;
  c->d_scratch = dev_alloc(c, std::max<size_t>(256, c->scratch_region * c->reg.size()));
  // per-medium receive outputs for the concurrent receives of small blocks
  c->rpart_cap = (int)std::min<int64_t>(nrhs, RPART_MAX_RHS);
  c->d_rpart = dev_alloc(c, std::max<size_t>(256, (size_t)c->rpart_nb * 2 * c->rpart_cap * sizeof(zd)));
  // right-hand-side-interleaved source and result of the block ILU(0) sweeps
  // ([n][Rp] each, Rp = nrhs rounded up to 16; the widest block used is 16)
  if (nrhs >= 2) {
    c->iluT_R = (int)((nrhs + 15) / 16 * 16);
    c->d_iluT = dev_alloc(c, (size_t)2 * c->iluT_R * c->ne * 2 * sizeof(zd));
  }
  c->nrhs_cap = nrhs;
  c->work_gen++;
}

// ------------------------------------------------------------------ special functions
// Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton iteration.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
      if (n == 1) { pn = z; pm = 1.0; }
      double dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
    double dp = n * (z * pn - pm) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// P_0..P_L at x
static void legendre_all(int L, double x, double *P) {
  P[0] = 1.0;
  if (L >= 1) P[1] = x;
  for (int n = 1; n < L; ++n) P[n + 1] = ((2.0 * n + 1.0) * x * P[n] - n * P[n - 1]) / (n + 1.0);
}

// spherical Hankel functions of the second kind h_0..h_L at complex z (upward recurrence)
static void hankel2_all(int L, cd z, cd *h) {
  const cd j(0.0, 1.0);
  cd e = std::exp(-j * z);
  h[0] = j * e / z;
  if (L >= 1) h[1] = e * (j / (z * z) - 1.0 / z);
  for (int n = 1; n < L; ++n) h[n + 1] = (2.0 * n + 1.0) / z * h[n] - h[n - 1];
}

static int64_t morton3(int i, int j, int k) {
  int64_t code = 0;
  for (int b = 0; b < 21; ++b) {
    code |= (int64_t)((i >> b) & 1) << (3 * b);
    code |= (int64_t)((j >> b) & 1) << (3 * b + 1);
    code |= (int64_t)((k >> b) & 1) << (3 * b + 2);
  }
  return code;
}
static inline int64_t ijk_key(int i, int j, int k) { return ((int64_t)i << 42) | ((int64_t)j << 21) | (int64_t)k; }

// ------------------------------------------------------------------ API: context
extern "C" sie_status sie_create(sie_ctx **out, int device, void *cuda_stream) {
  if (!out) return SIE_EINVAL;
  sie_ctx *c = new sie_ctx();
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete c;
    return SIE_ECUDA;
  }
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return SIE_ECUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return SIE_OK;
}

extern "C" void sie_destroy(sie_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  nn_free(c);
  graphs_free(c);
  for (auto &b : c->bufs) cudaFree(b.p);
  for (auto s : c->rstream) cudaStreamDestroy(s);
  for (auto e : c->ev_join) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->gm_hpin) cudaFreeHost(c->gm_hpin);
  if (c->gm_ev) cudaEventDestroy(c->gm_ev);
  if (c->gm_ev0) cudaEventDestroy(c->gm_ev0);
  if (c->gm_cs) cudaStreamDestroy(c->gm_cs);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" const char *sie_last_error(const sie_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

template <typename F>
static sie_status guard(sie_ctx *c, F &&f) {
  if (!c) return SIE_EINVAL;
  try {
    cudaSetDevice(c->device);
    f();
    return SIE_OK;
  } catch (const SieError &e) {
    c->last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    c->last_error = "host allocation failed";
    return SIE_ENOMEM;
  } catch (const std::exception &e) {
    c->last_error = e.what();
    return SIE_EINVAL;
  }
}

// ------------------------------------------------------------------ API: mesh
static void build_mesh(sie_ctx *c, const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                       const int32_t *treg, const double *media, int32_t nr, double freq) {
  SIE_REQUIRE(verts && tris && treg && media && nv > 0 && nt > 0 && nr > 0 && freq > 0, SIE_EINVAL,
              "sie_build_mesh: null pointer or non-positive size");
  SIE_REQUIRE(nt < (1 << 30) && nv < (1 << 30), SIE_EINVAL, "sie_build_mesh: mesh too large");
  c->nv = (int)nv;
  c->nt = (int)nt;
  c->nr = nr;
  c->freq = freq;
  c->k0 = 2.0 * PI * freq / 299792458.0;
  c->verts.assign(verts, verts + 3 * nv);
  c->tris.assign(tris, tris + 3 * nt);
  c->tri_reg.assign(treg, treg + 2 * nt);
  c->media.assign(media, media + 4 * nr);
  for (int64_t t = 0; t < nt; ++t) {
    for (int a = 0; a < 3; ++a)
      SIE_REQUIRE(tris[3 * t + a] >= 0 && tris[3 * t + a] < nv, SIE_EINVAL, "sie_build_mesh: vertex index out of range");
    for (int a = 0; a < 2; ++a)
      SIE_REQUIRE(treg[2 * t + a] >= 0 && treg[2 * t + a] < nr, SIE_EINVAL, "sie_build_mesh: region index out of range");
    SIE_REQUIRE(treg[2 * t] != treg[2 * t + 1], SIE_EINVAL, "sie_build_mesh: triangle with the same region on both sides");
  }
  // media
  c->kreg.resize(nr);
  c->etareg.resize(nr);
  for (int l = 0; l < nr; ++l) {
    cd eps(media[4 * l], media[4 * l + 1]), mu(media[4 * l + 2], media[4 * l + 3]);
    SIE_REQUIRE(std::isfinite(std::abs(eps)) && std::isfinite(std::abs(mu)) && std::abs(eps) > 0.0 &&
                    std::abs(mu) > 0.0,
                SIE_EINVAL, "sie_build_mesh: medium with zero or non-finite eps_r or mu_r");
    cd k = c->k0 * std::sqrt(eps * mu);
    SIE_REQUIRE(k.imag() <= 0.0, SIE_EINVAL, "sie_build_mesh: active medium (Im eps_r mu_r > 0)");
    cd eta = std::sqrt(mu / eps);
    if (eta.real() < 0) eta = -eta;
    c->kreg[l] = k;
    c->etareg[l] = eta;
  }
  // triangle geometry (same arithmetic order as the definition: mean, norms)
  c->area.resize(nt);
  c->normal.resize(3 * nt);
  c->centroid.resize(3 * nt);
  c->hmax.resize(nt);
  for (int64_t t = 0; t < nt; ++t) {
    const double *P[3];
    for (int a = 0; a < 3; ++a) P[a] = &verts[3 * tris[3 * t + a]];
    double e1[3], e2[3], cr[3];
    for (int x = 0; x < 3; ++x) {
      e1[x] = P[1][x] - P[0][x];
      e2[x] = P[2][x] - P[0][x];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double n2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    SIE_REQUIRE(n2 > 0, SIE_EINVAL, "sie_build_mesh: degenerate triangle");
    c->area[t] = 0.5 * n2;
    for (int x = 0; x < 3; ++x) {
      c->normal[3 * t + x] = cr[x] / (2.0 * c->area[t]);
      c->centroid[3 * t + x] = ((P[0][x] + P[1][x]) + P[2][x]) / 3.0;
    }
    double hm = 0;
    for (int a = 0; a < 3; ++a) {
      const double *A = P[a], *B = P[(a + 1) % 3];
      double dx = A[0] - B[0], dy = A[1] - B[1], dz = A[2] - B[2];
      hm = std::max(hm, std::sqrt((dx * dx + dy * dy) + dz * dz));
    }
    c->hmax[t] = hm;
  }
  // edges: sort (key, triangle) records
  struct Rec {
    int64_t key;
    int t, free_v, u, v;
  };
  std::vector<Rec> recs;
  recs.reserve(3 * nt);
  for (int t = 0; t < (int)nt; ++t) {
    int a = tris[3 * t], b = tris[3 * t + 1], cc = tris[3 * t + 2];
    int U[3] = {a, b, cc}, V[3] = {b, cc, a}, W[3] = {cc, a, b};
    for (int s = 0; s < 3; ++s) {
      int lo = std::min(U[s], V[s]), hi = std::max(U[s], V[s]);
      recs.push_back({((int64_t)lo << 32) | (int64_t)hi, t, W[s], U[s], V[s]});
    }
  }
  std::sort(recs.begin(), recs.end(), [](const Rec &x, const Rec &y) {
    return x.key < y.key || (x.key == y.key && x.t < y.t);
  });
  c->edge_v.clear();
  c->tp.clear();
  c->tm.clear();
  c->vp.clear();
  c->vm.clear();
  c->elen.clear();
  c->tri_edge.assign(3 * nt, -1);
  c->tri_free.assign(3 * nt, 0);
  c->tri_sign.assign(3 * nt, 0.0);
  c->emed_ptr.assign(1, 0);
  c->emed.clear();
  c->ejunc.clear();
  c->njunc = 0;
  std::vector<int> fillc(nt, 0);
  auto side = [&](int l, int t) { return treg[2 * t] == l ? 1.0 : -1.0; };
  size_t i = 0;
  while (i < recs.size()) {
    size_t j = i;
    while (j < recs.size() && recs[j].key == recs[i].key) ++j;
    size_t cnt = j - i;
    if (cnt >= 3) {
      // junction edge: each region touching it sees two of the triangles; one
      // unknown with per-triangle coefficients a_T, s_l(T1) a_T1 = -s_l(T2) a_T2
      // for every such region (continuity of that region's current across the edge)
      std::vector<int> ts;
      for (size_t q = i; q < j; ++q) ts.push_back(recs[q].t);
      std::vector<int> regs;
      for (int t : ts)
        for (int a = 0; a < 2; ++a)
          if (std::find(regs.begin(), regs.end(), (int)treg[2 * t + a]) == regs.end()) regs.push_back(treg[2 * t + a]);
      std::sort(regs.begin(), regs.end());
      std::vector<std::array<int, 3>> pr;  // (region, T1, T2)
      for (int l : regs) {
        std::vector<int> tl;
        for (int t : ts)
          if (treg[2 * t] == l || treg[2 * t + 1] == l) tl.push_back(t);
        SIE_REQUIRE(tl.size() == 2, SIE_EINVAL, "sie_build_mesh: junction edge where a region does not see two faces");
        pr.push_back({l, tl[0], tl[1]});
      }
      std::map<int, double> av;
      av[ts[0]] = 1.0;
      for (size_t it = 0; it < pr.size(); ++it)
        for (auto &q : pr) {
          const bool h1 = av.count(q[1]), h2 = av.count(q[2]);
          if (h1 && !h2) av[q[2]] = -side(q[0], q[1]) * side(q[0], q[2]) * av[q[1]];
          if (h2 && !h1) av[q[1]] = -side(q[0], q[1]) * side(q[0], q[2]) * av[q[2]];
        }
      SIE_REQUIRE(av.size() == ts.size(), SIE_EINVAL, "sie_build_mesh: junction faces not connected through regions");
      for (auto &q : pr)
        SIE_REQUIRE(side(q[0], q[1]) * av[q[1]] == -side(q[0], q[2]) * av[q[2]], SIE_EINVAL,
                    "sie_build_mesh: inconsistent junction continuity constraints");
      int e = (int)c->tp.size();
      int lo = (int)(recs[i].key >> 32), hi = (int)(recs[i].key & 0xffffffff);
      c->edge_v.push_back(lo);
      c->edge_v.push_back(hi);
      c->tp.push_back(recs[i].t);
      c->tm.push_back(recs[i + 1].t);
      c->vp.push_back(recs[i].free_v);
      c->vm.push_back(recs[i + 1].free_v);
      double dx = verts[3 * hi] - verts[3 * lo], dy = verts[3 * hi + 1] - verts[3 * lo + 1],
             dz = verts[3 * hi + 2] - verts[3 * lo + 2];
      c->elen.push_back(std::sqrt(dx * dx + dy * dy + dz * dz));
      for (size_t q = i; q < j; ++q) {
        int t = recs[q].t;
        int f = fillc[t]++;
        c->tri_edge[3 * t + f] = e;
        c->tri_free[3 * t + f] = recs[q].free_v;
        c->tri_sign[3 * t + f] = av[t];
      }
      for (auto &q : pr) c->emed.push_back(q);
      c->emed_ptr.push_back((int)c->emed.size());
      c->ejunc.push_back(1);
      c->njunc++;
      i = j;
      continue;
    }
    if (cnt == 2) {
      const Rec &r1 = recs[i], &r2 = recs[i + 1];
      SIE_REQUIRE(treg[2 * r1.t] == treg[2 * r2.t] && treg[2 * r1.t + 1] == treg[2 * r2.t + 1], SIE_EINVAL,
                  "sie_build_mesh: edge shared by triangles of different surfaces");
      SIE_REQUIRE(r1.u == r2.v && r1.v == r2.u, SIE_EINVAL,
                  "sie_build_mesh: inconsistent triangle orientation across an edge");
      int e = (int)c->tp.size();
      // the two media of the surface, each with the pair (T+, T-)
      c->emed.push_back({(int)treg[2 * r1.t], r1.t, r2.t});
      c->emed.push_back({(int)treg[2 * r1.t + 1], r1.t, r2.t});
      c->emed_ptr.push_back((int)c->emed.size());
      c->ejunc.push_back(0);
      int lo = (int)(r1.key >> 32), hi = (int)(r1.key & 0xffffffff);
      c->edge_v.push_back(lo);
      c->edge_v.push_back(hi);
      c->tp.push_back(r1.t);
      c->tm.push_back(r2.t);
      c->vp.push_back(r1.free_v);
      c->vm.push_back(r2.free_v);
      double dx = verts[3 * hi] - verts[3 * lo], dy = verts[3 * hi + 1] - verts[3 * lo + 1],
             dz = verts[3 * hi + 2] - verts[3 * lo + 2];
      c->elen.push_back(std::sqrt(dx * dx + dy * dy + dz * dz));
      const Rec *rr[2] = {&r1, &r2};
      for (int s = 0; s < 2; ++s) {
        int t = rr[s]->t;
        int f = fillc[t]++;
        c->tri_edge[3 * t + f] = e;
        c->tri_free[3 * t + f] = rr[s]->free_v;
        c->tri_sign[3 * t + f] = s == 0 ? 1.0 : -1.0;
      }
    }
    i = j;
  }
  c->ne = (int)c->tp.size();
  SIE_REQUIRE(c->ne > 0, SIE_EINVAL, "sie_build_mesh: no RWG edge (open or empty mesh)");
  c->have_mesh = true;
  c->have_tree = c->have_fill = false;
}

extern "C" sie_status sie_build_mesh(sie_ctx *c, const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                     const int32_t *tri_regions, const double *media, int32_t nr, double freq_hz,
                                     int64_t *n_rwg_out) {
  return guard(c, [&] {
    SIE_REQUIRE(!c->have_mesh, SIE_ESTATE, "sie_build_mesh: context already holds a mesh");
    build_mesh(c, verts, nv, tris, nt, tri_regions, media, nr, freq_hz);
    if (n_rwg_out) *n_rwg_out = c->ne;
  });
}

// ------------------------------------------------------------------ API: tree + MLFMM tables
static int trunc_L(double kr, double a, double d0) {
  double kd = kr * std::sqrt(3.0) * a;
  double L = kd + 1.8 * std::pow(d0, 2.0 / 3.0) * std::pow(kd, 1.0 / 3.0);
  return std::max(2, (int)std::ceil(L));
}

struct Dirs {
  int L, K;
  std::vector<double> d;  // [K][9]
  std::vector<double> w;  // [K]
};
static Dirs make_dirs(int L) {
  Dirs D;
  D.L = L;
  int nth = L + 1, nph = 2 * L + 2;
  D.K = nth * nph;
  std::vector<double> x, wx;
  gauss_legendre(nth, x, wx);
  D.d.resize(9 * D.K);
  D.w.resize(D.K);
  for (int it = 0; it < nth; ++it) {
    double ct = x[it], st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    for (int jp = 0; jp < nph; ++jp) {
      double ph = 2.0 * PI * jp / nph, cp = std::cos(ph), sp = std::sin(ph);
      int k = it * nph + jp;
      double *o = &D.d[9 * k];
      o[0] = st * cp; o[1] = st * sp; o[2] = ct;          // khat
      o[3] = ct * cp; o[4] = ct * sp; o[5] = -st;         // theta_hat
      o[6] = -sp;     o[7] = cp;      o[8] = 0.0;         // phi_hat
      D.w[k] = wx[it] * 2.0 * PI / nph;
    }
  }
  return D;
}

static void setup_tree(sie_ctx *c, int levels, double digits) {
  SIE_REQUIRE(levels >= 2 && levels <= 12, SIE_EINVAL, "mlfmm_setup: levels must be in [2, 12]");
  SIE_REQUIRE(digits > 0 && digits < 16, SIE_EINVAL, "mlfmm_setup: digits must be in (0, 16)");
  c->levels = levels;
  c->digits = digits;
  const int ne = c->ne;
  // root cube
  double lo[3], hi[3];
  for (int x = 0; x < 3; ++x) lo[x] = hi[x] = c->verts[x];
  for (int v = 0; v < c->nv; ++v)
    for (int x = 0; x < 3; ++x) {
      lo[x] = std::min(lo[x], c->verts[3 * v + x]);
      hi[x] = std::max(hi[x], c->verts[3 * v + x]);
    }
  double ext = 0, centre[3];
  for (int x = 0; x < 3; ++x) {
    centre[x] = (lo[x] + hi[x]) * 0.5;
    ext = std::max(ext, hi[x] - lo[x]);
  }
  c->D = ext * 1.0009765625;
  int nleaf = 1 << (levels - 1);
  c->hleaf = c->D / nleaf;
  for (int x = 0; x < 3; ++x) c->origin[x] = centre[x] - 0.5 * c->D;
  c->eijk.resize(3 * ne);
  for (int e = 0; e < ne; ++e) {
    const double *A = &c->verts[3 * c->edge_v[2 * e]], *B = &c->verts[3 * c->edge_v[2 * e + 1]];
    for (int x = 0; x < 3; ++x) {
      double mid = (A[x] + B[x]) * 0.5;
      int q = (int)std::floor((mid - c->origin[x]) / c->hleaf);
      c->eijk[3 * e + x] = std::min(std::max(q, 0), nleaf - 1);
    }
  }
  // internal order: (colour, Morton, edge)
  std::vector<int64_t> key(ne);
  for (int e = 0; e < ne; ++e) {
    int i = c->eijk[3 * e], j = c->eijk[3 * e + 1], k = c->eijk[3 * e + 2];
    int col = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    key[e] = ((int64_t)col << 60) | morton3(i, j, k);
  }
  c->perm.resize(ne);
  for (int e = 0; e < ne; ++e) c->perm[e] = e;
  std::stable_sort(c->perm.begin(), c->perm.end(), [&](int a, int b) { return key[a] < key[b]; });
  c->inv.resize(ne);
  for (int p = 0; p < ne; ++p) c->inv[c->perm[p]] = p;
  // global leaf boxes in internal order
  c->leaf_start.clear();
  c->leaf_ijk.clear();
  std::vector<int> ebox(ne);  // leaf box of internal edge p
  for (int p = 0; p < ne; ++p) {
    int e = c->perm[p];
    if (p == 0 || key[e] != key[c->perm[p - 1]]) {
      c->leaf_start.push_back(p);
      for (int x = 0; x < 3; ++x) c->leaf_ijk.push_back(c->eijk[3 * e + x]);
    }
    ebox[p] = (int)c->leaf_start.size() - 1;
  }
  int nlb = (int)c->leaf_start.size();
  c->leaf_start.push_back(ne);
  std::unordered_map<int64_t, int> leaf_map;
  for (int b = 0; b < nlb; ++b) leaf_map[ijk_key(c->leaf_ijk[3 * b], c->leaf_ijk[3 * b + 1], c->leaf_ijk[3 * b + 2])] = b;
  // near pattern: rows in internal order, columns sorted
  std::vector<std::vector<int>> nb_of(nlb);
  for (int b = 0; b < nlb; ++b) {
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          auto it = leaf_map.find(ijk_key(c->leaf_ijk[3 * b] + dx, c->leaf_ijk[3 * b + 1] + dy, c->leaf_ijk[3 * b + 2] + dz));
          if (it != leaf_map.end()) nb_of[b].push_back(it->second);
        }
    std::sort(nb_of[b].begin(), nb_of[b].end(), [&](int x, int y) { return c->leaf_start[x] < c->leaf_start[y]; });
  }
  c->row_ptr.assign(ne + 1, 0);
  for (int p = 0; p < ne; ++p) {
    int cnt = 0;
    for (int b : nb_of[ebox[p]]) cnt += c->leaf_start[b + 1] - c->leaf_start[b];
    c->row_ptr[p + 1] = c->row_ptr[p] + cnt;
  }
  SIE_REQUIRE((int64_t)c->row_ptr[ne] < ((int64_t)1 << 31), SIE_EINVAL, "mlfmm_setup: near field too large (more levels needed)");
  c->col.resize(c->row_ptr[ne]);
  for (int p = 0; p < ne; ++p) {
    int o = c->row_ptr[p];
    for (int b : nb_of[ebox[p]])
      for (int q = c->leaf_start[b]; q < c->leaf_start[b + 1]; ++q) c->col[o++] = q;
  }

  // ---------------- per medium
  c->reg.assign(c->nr, RegionHost());
  int leaf = levels - 1;
  for (int l = 0; l < c->nr; ++l) {
    RegionHost &R = c->reg[l];
    R.id = l;
    R.k = c->kreg[l];
    R.eta = c->etareg[l];
    std::vector<int> basis_gbox;
    for (int p = 0; p < ne; ++p) {
      int e = c->perm[p];
      const bool junction = c->ejunc[e] != 0;
      for (int q = c->emed_ptr[e]; q < c->emed_ptr[e + 1]; ++q) {
        const auto &E = c->emed[q];
        if (E[0] != l) continue;
        const double s1 = c->tri_reg[2 * E[1]] == l ? 1.0 : -1.0, s2 = c->tri_reg[2 * E[2]] == l ? 1.0 : -1.0;
        R.basis_p.push_back(p);
        R.basis_sign.push_back(junction ? 1 : (int)s1);
        R.ptri.push_back(E[1]);
        R.ptri.push_back(E[2]);
        R.psg.push_back(junction ? s1 : 1.0);
        R.psg.push_back(junction ? s2 : 1.0);
        basis_gbox.push_back(ebox[p]);
      }
    }
    R.nb = (int)R.basis_p.size();
    R.lev.assign(levels, LevelHost());
    for (int lv = 0; lv < levels; ++lv) {
      R.lev[lv].lev = lv;
      R.lev[lv].a = c->D / (double)(1 << lv);
    }
    if (R.nb == 0) continue;
    // leaf level: boxes in internal order
    LevelHost &LL = R.lev[leaf];
    std::vector<int> basis_box(R.nb);
    for (int i = 0; i < R.nb; ++i) {
      if (i == 0 || basis_gbox[i] != basis_gbox[i - 1]) {
        R.box_start.push_back(i);
        int g = basis_gbox[i];
        for (int x = 0; x < 3; ++x) LL.ijk.push_back(c->leaf_ijk[3 * g + x]);
      }
      basis_box[i] = (int)R.box_start.size() - 1;
    }
    LL.nbox = (int)R.box_start.size();
    R.box_start.push_back(R.nb);
    // coarser levels (Morton order)
    for (int lv = leaf - 1; lv >= 1; --lv) {
      LevelHost &C = R.lev[lv + 1], &P = R.lev[lv];
      std::vector<std::pair<int64_t, int>> keys;  // (morton, child)
      for (int b = 0; b < C.nbox; ++b)
        keys.push_back({morton3(C.ijk[3 * b] >> 1, C.ijk[3 * b + 1] >> 1, C.ijk[3 * b + 2] >> 1), b});
      std::sort(keys.begin(), keys.end());
      C.parent.assign(C.nbox, -1);
      C.oct.assign(C.nbox, 0);
      P.ch_ptr.assign(1, 0);
      for (size_t s = 0; s < keys.size(); ++s) {
        int b = keys[s].second;
        if (s == 0 || keys[s].first != keys[s - 1].first) {
          for (int x = 0; x < 3; ++x) P.ijk.push_back(C.ijk[3 * b + x] >> 1);
          P.ch_ptr.push_back(P.ch_ptr.back());
        }
        int pb = (int)P.ch_ptr.size() - 2;
        C.parent[b] = pb;
        C.oct[b] = (C.ijk[3 * b] & 1) | ((C.ijk[3 * b + 1] & 1) << 1) | ((C.ijk[3 * b + 2] & 1) << 2);
        P.ch_idx.push_back(b);
        P.ch_ptr.back()++;
      }
      P.nbox = (int)P.ch_ptr.size() - 1;
    }
    // interaction lists, levels 2..leaf
    for (int lv = 2; lv <= leaf; ++lv) {
      LevelHost &B = R.lev[lv], &P = R.lev[lv - 1];
      std::unordered_map<int64_t, int> pmap;
      for (int pb = 0; pb < P.nbox; ++pb) pmap[ijk_key(P.ijk[3 * pb], P.ijk[3 * pb + 1], P.ijk[3 * pb + 2])] = pb;
      std::map<int, int> slot_of;
      B.il_ptr.assign(1, 0);
      for (int b = 0; b < B.nbox; ++b) {
        int pb = B.parent[b];
        for (int dx = -1; dx <= 1; ++dx)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
              auto it = pmap.find(ijk_key(P.ijk[3 * pb] + dx, P.ijk[3 * pb + 1] + dy, P.ijk[3 * pb + 2] + dz));
              if (it == pmap.end()) continue;
              int nbp = it->second;
              for (int s = P.ch_ptr[nbp]; s < P.ch_ptr[nbp + 1]; ++s) {
                int b2 = P.ch_idx[s];
                int d[3];
                int far = 0;
                for (int x = 0; x < 3; ++x) {
                  d[x] = B.ijk[3 * b + x] - B.ijk[3 * b2 + x];
                  far = std::max(far, std::abs(d[x]));
                }
                if (far < 2) continue;
                int code = (d[0] + 3) * 49 + (d[1] + 3) * 7 + (d[2] + 3);
                auto si = slot_of.find(code);
                int slot;
                if (si == slot_of.end()) {
                  slot = (int)B.slot_code.size();
                  slot_of[code] = slot;
                  B.slot_code.push_back(code);
                } else {
                  slot = si->second;
                }
                B.il_src.push_back(b2);
                B.il_slot.push_back(slot);
              }
            }
        B.il_ptr.push_back((int)B.il_src.size());
      }
    }
    R.top = leaf;
    for (int lv = 2; lv <= leaf; ++lv)
      if (!R.lev[lv].il_src.empty()) {
        R.top = lv;
        break;
      }
    // directions and tables; the truncation follows |k|: in a lossy medium
    // the addition theorem converges at the rate set by the modulus of k d,
    // not its real part (a metal's k is nearly imaginary)
    double kr = std::abs(R.k);
    for (int lv = R.top; lv <= leaf; ++lv) {
      LevelHost &B = R.lev[lv];
      B.L = trunc_L(kr, B.a, digits);
    }
    std::vector<Dirs> dirs(levels);
    for (int lv = R.top; lv <= leaf; ++lv) {
      dirs[lv] = make_dirs(R.lev[lv].L);
      R.lev[lv].K = dirs[lv].K;
    }
    cd kc = R.k;
    cd pref = kc * kc / (16.0 * PI * PI);
    for (int lv = R.top; lv <= leaf; ++lv) {
      LevelHost &B = R.lev[lv];
      const Dirs &Dd = dirs[lv];
      int K = Dd.K, L = Dd.L;
      B.d_dirs = dev_upload(c, Dd.d);
      {  // theta_hat, phi_hat per direction for the Cartesian <-> (theta, phi) steps
        std::vector<double> tp(6 * (size_t)K);
        std::vector<float> tpf(6 * (size_t)K);
        for (int k = 0; k < K; ++k)
          for (int q = 0; q < 6; ++q) {
            tp[6 * k + q] = Dd.d[9 * k + 3 + q];
            tpf[6 * k + q] = (float)Dd.d[9 * k + 3 + q];
          }
        B.d_tp64 = dev_upload(c, tp);
        B.d_tp32 = dev_upload(c, tpf);
      }
      // translators (weights and constants folded in)
      int ns = (int)B.slot_code.size();
      std::vector<cd> T((size_t)std::max(ns, 1) * K);
      std::vector<cd> h(L + 1);
      std::vector<double> Pl(L + 1);
      for (int s = 0; s < ns; ++s) {
        int code = B.slot_code[s];
        int d[3] = {code / 49 - 3, (code / 7) % 7 - 3, code % 7 - 3};
        double X[3] = {d[0] * B.a, d[1] * B.a, d[2] * B.a};
        double Xn = std::sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
        hankel2_all(L, kc * Xn, h.data());
        std::vector<cd> coef(L + 1);
        cd mj(1.0, 0.0);
        for (int n = 0; n <= L; ++n) {
          coef[n] = mj * (2.0 * n + 1.0) * h[n];
          mj *= cd(0.0, -1.0);
        }
        for (int k = 0; k < K; ++k) {
          const double *kh = &Dd.d[9 * k];
          double ct = (kh[0] * X[0] + kh[1] * X[1] + kh[2] * X[2]) / Xn;
          legendre_all(L, ct, Pl.data());
          cd acc = 0.0;
          for (int n = 0; n <= L; ++n) acc += coef[n] * Pl[n];
          T[(size_t)s * K + k] = pref * Dd.w[k] * acc;
        }
      }
      B.d_T64 = dev_upload(c, T);
      std::vector<std::complex<float>> Tf(T.size());
      for (size_t q = 0; q < T.size(); ++q) Tf[q] = std::complex<float>((float)T[q].real(), (float)T[q].imag());
      B.d_T32 = dev_upload(c, Tf);
      B.d_il_ptr = dev_upload(c, B.il_ptr);
      B.d_il_src = dev_upload(c, B.il_src);
      B.d_il_slot = dev_upload(c, B.il_slot);
      {
        // sibling groups: the union of the members' interaction lists, per source
        // the members that take it and their translator slots
        LevelHost &Pg = R.lev[lv - 1];
        std::vector<int> gptr(1, 0), gbox, gent;
        for (int pb = 0; pb < Pg.nbox; ++pb) {
          const int m = Pg.ch_ptr[pb + 1] - Pg.ch_ptr[pb];
          if (m == 0) continue;
          SIE_REQUIRE(m <= 8, SIE_EINVAL, "octree: more than 8 children");
          std::map<int, std::array<int, 8>> ent;
          for (int u = 0; u < 8; ++u) gbox.push_back(u < m ? Pg.ch_idx[Pg.ch_ptr[pb] + u] : -1);
          for (int u = 0; u < m; ++u) {
            const int b = Pg.ch_idx[Pg.ch_ptr[pb] + u];
            for (int e = B.il_ptr[b]; e < B.il_ptr[b + 1]; ++e) {
              auto it = ent.find(B.il_src[e]);
              if (it == ent.end()) {
                std::array<int, 8> a;
                a.fill(-1);
                it = ent.emplace(B.il_src[e], a).first;
              }
              it->second[u] = B.il_slot[e];
            }
          }
          for (auto &kv : ent) {
            int mask = 0;
            for (int u = 0; u < 8; ++u)
              if (kv.second[u] >= 0) mask |= 1 << u;
            gent.push_back(kv.first);
            gent.push_back(mask);
            for (int u = 0; u < 8; ++u) gent.push_back(std::max(0, kv.second[u]));
          }
          gptr.push_back((int)(gent.size() / 10));
        }
        B.ngroups = (int)gptr.size() - 1;
        B.max_group_entries = 0;
        for (int q = 0; q < B.ngroups; ++q) B.max_group_entries = std::max(B.max_group_entries, gptr[q + 1] - gptr[q]);
        B.d_grp_ptr = dev_upload(c, gptr);
        B.d_grp_box = dev_upload(c, gbox);
        B.d_grp_ent = dev_upload(c, gent.empty() ? std::vector<int>(10, 0) : gent);
      }
      // shifts between this level (parent) and its children
      if (lv < leaf) {
        std::vector<cd> up(8 * K), dn(8 * K);
        const cd j(0.0, 1.0);
        for (int o = 0; o < 8; ++o) {
          double dl[3] = {B.a * 0.25 * (2 * (o & 1) - 1), B.a * 0.25 * (2 * ((o >> 1) & 1) - 1),
                          B.a * 0.25 * (2 * ((o >> 2) & 1) - 1)};
          for (int k = 0; k < K; ++k) {
            const double *kh = &Dd.d[9 * k];
            double kd = kh[0] * dl[0] + kh[1] * dl[1] + kh[2] * dl[2];
            up[o * K + k] = std::exp(j * kc * kd);
            dn[o * K + k] = std::exp(-j * kc * kd);
          }
        }
        B.d_up64 = dev_upload(c, up);
        B.d_dn64 = dev_upload(c, dn);
        std::vector<std::complex<float>> uf(8 * K), df(8 * K);
        for (int q = 0; q < 8 * K; ++q) {
          uf[q] = std::complex<float>((float)up[q].real(), (float)up[q].imag());
          df[q] = std::complex<float>((float)dn[q].real(), (float)dn[q].imag());
        }
        B.d_up32 = dev_upload(c, uf);
        B.d_dn32 = dev_upload(c, df);
        // Exact separable interpolation from level lv+1, applied to Cartesian
        // components (band-limited to degree Lc on the sphere):
        //  phi:   trigonometric interpolation, Nc = 2Lc+2 uniform samples -> Np,
        //         Phi[jp][jc] = (1 + 2 sum_{m=1..Lc} cos m(phi_p - phi_c)) / Nc;
        //  theta: along the meridian through phi and phi+pi the function is a
        //         trigonometric polynomial of degree Lc; its even part is a
        //         polynomial in cos(theta) and its odd part sin(theta) times one,
        //         both interpolated by the Lagrange basis l_i on the child's
        //         Gauss-Legendre nodes:
        //         h(theta_p) = sum_i l_i(x_p) [ (1+s)/2 g_i(phi) + (1-s)/2 g_i(phi+pi) ],
        //         s = sin(theta_p) / sin(theta_i).
        const Dirs &Dc = dirs[lv + 1];
        int Lc = Dc.L, Nc = 2 * Lc + 2, Np = 2 * L + 2, nthc = Lc + 1, nthp = L + 1;
        std::vector<double> Phi((size_t)Np * Nc), Thp((size_t)nthp * nthc), Thm((size_t)nthp * nthc);
        for (int jp = 0; jp < Np; ++jp)
          for (int jc = 0; jc < Nc; ++jc) {
            double dphi = 2.0 * PI * jp / Np - 2.0 * PI * jc / Nc;
            double s = 1.0;
            for (int m = 1; m <= Lc; ++m) s += 2.0 * std::cos(m * dphi);
            Phi[(size_t)jp * Nc + jc] = s / Nc;
          }
        std::vector<double> xc(nthc), xp(nthp);
        for (int i = 0; i < nthc; ++i) xc[i] = Dc.d[9 * (i * Nc) + 2];
        for (int i = 0; i < nthp; ++i) xp[i] = Dd.d[9 * (i * Np) + 2];
        for (int p = 0; p < nthp; ++p)
          for (int i = 0; i < nthc; ++i) {
            double li = 1.0;
            for (int q = 0; q < nthc; ++q)
              if (q != i) li *= (xp[p] - xc[q]) / (xc[i] - xc[q]);
            double s = std::sqrt(1.0 - xp[p] * xp[p]) / std::sqrt(1.0 - xc[i] * xc[i]);
            Thp[(size_t)p * nthc + i] = 0.5 * li * (1.0 + s);
            Thm[(size_t)p * nthc + i] = 0.5 * li * (1.0 - s);
          }
        auto upf = [&](const std::vector<double> &v, void *&d64, void *&d32) {
          d64 = dev_upload(c, v);
          std::vector<float> f(v.size());
          for (size_t q = 0; q < v.size(); ++q) f[q] = (float)v[q];
          d32 = dev_upload(c, f);
        };
        upf(Phi, B.d_Phi64, B.d_Phi32);
        upf(Thp, B.d_Thp64, B.d_Thp32);
        upf(Thm, B.d_Thm64, B.d_Thm32);
        B.d_ch_ptr = dev_upload(c, B.ch_ptr);
        B.d_ch_idx = dev_upload(c, B.ch_idx);
      }
      if (lv > R.top) {
        B.d_oct = dev_upload(c, B.oct);
        B.d_parent = dev_upload(c, B.parent);
      }
    }
    // leaf tables
    R.d_basis_p = dev_upload(c, R.basis_p);
    R.d_basis_sign = dev_upload(c, R.basis_sign);
    R.d_ptri = dev_upload(c, R.ptri);
    R.d_psg = dev_upload(c, R.psg);
    R.d_box_start = dev_upload(c, R.box_start);
    R.max_leaf = 0;
    for (size_t b = 0; b + 1 < R.box_start.size(); ++b)
      R.max_leaf = std::max(R.max_leaf, R.box_start[b + 1] - R.box_start[b]);
    R.d_basis_box = dev_upload(c, basis_box);
    std::vector<double> cen(3 * LL.nbox);
    for (int b = 0; b < LL.nbox; ++b)
      for (int x = 0; x < 3; ++x) cen[3 * b + x] = c->origin[x] + (LL.ijk[3 * b + x] + 0.5) * c->hleaf;
    R.d_box_centre = dev_upload(c, cen);
  }
  // receive map: each basis lies on one interface, so its far field comes from
  // (at most) two media; per basis the positions of its rows in the
  // concatenated per-medium receive outputs, lower medium first (-1: none)
  {
    std::vector<int> rmap((size_t)2 * ne, -1);
    int off = 0;
    bool two = true;  // junction bases lie in more than two media: they receive one medium at a time
    for (auto &R : c->reg) {
      R.rpart_off = off;
      for (int i = 0; i < R.nb; ++i) {
        const int p = R.basis_p[i];
        if (rmap[2 * (size_t)p + 1] >= 0) {
          two = false;
          continue;
        }
        rmap[2 * (size_t)p + (rmap[2 * (size_t)p] < 0 ? 0 : 1)] = off + i;
      }
      off += R.nb;
    }
    c->rpart_nb = off;
    if (two) c->d_rmap = dev_upload(c, rmap);
  }
  c->have_tree = true;
}

extern "C" sie_status mlfmm_setup(sie_ctx *c, const sie_mlfmm_opts *o) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_mesh, SIE_ESTATE, "mlfmm_setup: call sie_build_mesh first");
    SIE_REQUIRE(!c->have_tree, SIE_ESTATE, "mlfmm_setup: already set up");
    SIE_REQUIRE(o, SIE_EINVAL, "mlfmm_setup: null options");
    setup_tree(c, o->levels, o->digits);
  });
}

// ------------------------------------------------------------------ ILU(0), 2x2 blocks, box-colour order
static inline void inv2(const cd *a, cd *o, bool &ok) {
  cd det = a[0] * a[3] - a[1] * a[2];
  if (std::abs(det) == 0.0 || !std::isfinite(std::abs(det))) {
    ok = false;
    return;
  }
  o[0] = a[3] / det;
  o[1] = -a[1] / det;
  o[2] = -a[2] / det;
  o[3] = a[0] / det;
}
static inline void mul2(const cd *a, const cd *b, cd *o) {
  cd r0 = a[0] * b[0] + a[1] * b[2], r1 = a[0] * b[1] + a[1] * b[3];
  cd r2 = a[2] * b[0] + a[3] * b[2], r3 = a[2] * b[1] + a[3] * b[3];
  o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3;
}

static void build_ilu(sie_ctx *c) {
  const int ne = c->ne;
  const int64_t nnz = c->row_ptr[ne];
  std::vector<cd> F((size_t)nnz * 4);
  SIE_CUDA(cudaMemcpy(F.data(), c->d_near64, (size_t)nnz * 4 * sizeof(cd), cudaMemcpyDeviceToHost));
  if (c->form == 4)  // ICTF: the near matrix of the system is D N (rows of block row i by D_i)
    for (int i = 0; i < ne; ++i)
      for (int e = c->row_ptr[i]; e < c->row_ptr[i + 1]; ++e) {
        F[4 * (size_t)e] *= c->rowscale[2 * (size_t)i];
        F[4 * (size_t)e + 1] *= c->rowscale[2 * (size_t)i];
        F[4 * (size_t)e + 2] *= c->rowscale[2 * (size_t)i + 1];
        F[4 * (size_t)e + 3] *= c->rowscale[2 * (size_t)i + 1];
      }
  std::vector<int> diag(ne, -1);
  for (int i = 0; i < ne; ++i)
    for (int e = c->row_ptr[i]; e < c->row_ptr[i + 1]; ++e)
      if (c->col[e] == i) diag[i] = e;
  int nlb = (int)c->leaf_start.size() - 1;
  std::vector<int> bcol(nlb);
  std::vector<int> cptr(9, 0);
  for (int b = 0; b < nlb; ++b) {
    bcol[b] = (c->leaf_ijk[3 * b] & 1) | ((c->leaf_ijk[3 * b + 1] & 1) << 1) | ((c->leaf_ijk[3 * b + 2] & 1) << 2);
    cptr[bcol[b] + 1]++;
  }
  for (int q = 0; q < 8; ++q) cptr[q + 1] += cptr[q];
  // boxes are already in colour order (internal order is colour-major)
  std::vector<cd> Dinv((size_t)ne * 4);
  std::atomic<bool> ok(true);
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  for (int col = 0; col < 8; ++col) {
    std::atomic<int> next(cptr[col]);
    auto work = [&]() {
      std::vector<int> where(ne, -1);
      for (;;) {
        int b = next.fetch_add(1);
        if (b >= cptr[col + 1]) break;
        for (int i = c->leaf_start[b]; i < c->leaf_start[b + 1]; ++i) {
          int s = c->row_ptr[i], e = c->row_ptr[i + 1];
          for (int q = s; q < e; ++q) where[c->col[q]] = q;
          for (int q = s; q < e && c->col[q] < i; ++q) {
            int k = c->col[q];
            cd m[4];
            mul2(&F[4 * (size_t)q], &Dinv[4 * (size_t)k], m);
            for (int x = 0; x < 4; ++x) F[4 * (size_t)q + x] = m[x];
            for (int r = diag[k] + 1; r < c->row_ptr[k + 1]; ++r) {
              int w = where[c->col[r]];
              if (w < 0) continue;
              cd u[4];
              mul2(m, &F[4 * (size_t)r], u);
              for (int x = 0; x < 4; ++x) F[4 * (size_t)w + x] -= u[x];
            }
          }
          bool good = true;
          inv2(&F[4 * (size_t)diag[i]], &Dinv[4 * (size_t)i], good);
          if (!good) ok = false;
          for (int q = s; q < e; ++q) where[c->col[q]] = -1;
        }
      }
    };
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nth; ++t) th.emplace_back(work);
    for (auto &t : th) t.join();
    SIE_REQUIRE(ok, SIE_EZEROPIVOT, "ILU(0): singular 2x2 diagonal block");
  }
  // apply structures
  std::vector<int> ebox(ne);
  for (int b = 0; b < nlb; ++b)
    for (int p = c->leaf_start[b]; p < c->leaf_start[b + 1]; ++p) ebox[p] = b;
  std::vector<int> lo_ptr(1, 0), up_ptr(1, 0), lo_col, up_col;
  std::vector<cd> lo_val, up_val;
  int maxb = 0;
  for (int b = 0; b < nlb; ++b) maxb = std::max(maxb, c->leaf_start[b + 1] - c->leaf_start[b]);
  for (int i = 0; i < ne; ++i) {
    int bi = ebox[i];
    for (int q = c->row_ptr[i]; q < c->row_ptr[i + 1]; ++q) {
      int k = c->col[q];
      const cd *v = &F[4 * (size_t)q];
      if (ebox[k] == bi) continue;
      if (k < i) {
        lo_col.push_back(k);
        for (int x = 0; x < 4; ++x) lo_val.push_back(v[x]);
      } else {
        up_col.push_back(k);
        for (int x = 0; x < 4; ++x) up_val.push_back(v[x]);
      }
    }
    lo_ptr.push_back((int)lo_col.size());
    up_ptr.push_back((int)up_col.size());
  }
  // in-box inverses, row-major blocks per box: X = L_bb^{-1} below the diagonal
  // (unit lower, X_jj = I), Y = U_bb^{-1} on and above it, by block substitution
  std::vector<int64_t> tloff(nlb + 1, 0), tuoff(nlb + 1, 0);
  for (int b = 0; b < nlb; ++b) {
    int64_t n = c->leaf_start[b + 1] - c->leaf_start[b];
    tloff[b + 1] = tloff[b] + n * (n - 1) / 2;
    tuoff[b + 1] = tuoff[b] + n * (n + 1) / 2;
  }
  std::vector<cd> tl((size_t)tloff[nlb] * 4), tu((size_t)tuoff[nlb] * 4);
  {
    std::atomic<int> next(0);
    auto work = [&]() {
      std::vector<cd> A, Xv;
      for (;;) {
        int b = next.fetch_add(1);
        if (b >= nlb) break;
        const int s0 = c->leaf_start[b], n = c->leaf_start[b + 1] - s0;
        A.assign((size_t)n * n * 4, cd(0.0));
        for (int i = s0; i < s0 + n; ++i)
          for (int q = c->row_ptr[i]; q < c->row_ptr[i + 1]; ++q) {
            int k = c->col[q];
            if (k < s0 || k >= s0 + n) continue;
            for (int x = 0; x < 4; ++x) A[((size_t)(i - s0) * n + (k - s0)) * 4 + x] = F[4 * (size_t)q + x];
          }
        Xv.assign((size_t)n * n * 4, cd(0.0));
        cd *X = Xv.data();
        auto blk = [&](cd *M, int i, int j) { return M + ((size_t)i * n + j) * 4; };
        for (int j = 0; j < n; ++j) {
          // column j of L^{-1}: X_ij = -sum_{j<=k<i} L_ik X_kj, X_jj = I (implicit)
          for (int i = j + 1; i < n; ++i) {
            cd acc[4] = {-A[((size_t)i * n + j) * 4], -A[((size_t)i * n + j) * 4 + 1],
                         -A[((size_t)i * n + j) * 4 + 2], -A[((size_t)i * n + j) * 4 + 3]};
            for (int k = j + 1; k < i; ++k) {
              cd u[4];
              mul2(blk(A.data(), i, k), blk(X, k, j), u);
              for (int x = 0; x < 4; ++x) acc[x] -= u[x];
            }
            for (int x = 0; x < 4; ++x) blk(X, i, j)[x] = acc[x];
          }
          // column j of U^{-1}: Y_jj = D_j^{-1}, Y_ij = -D_i^{-1} sum_{i<k<=j} U_ik Y_kj
          for (int x = 0; x < 4; ++x) blk(X, j, j)[x] = Dinv[4 * (size_t)(s0 + j) + x];
          for (int i = j - 1; i >= 0; --i) {
            cd acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int k = i + 1; k <= j; ++k) {
              cd u[4];
              mul2(blk(A.data(), i, k), blk(X, k, j), u);
              for (int x = 0; x < 4; ++x) acc[x] -= u[x];
            }
            mul2(&Dinv[4 * (size_t)(s0 + i)], acc, blk(X, i, j));
          }
        }
        // pack by rows
        for (int i = 0; i < n; ++i) {
          cd *dl = &tl[(size_t)(tloff[b] + (int64_t)i * (i - 1) / 2) * 4];
          for (int j = 0; j < i; ++j)
            for (int x = 0; x < 4; ++x) dl[4 * j + x] = blk(X, i, j)[x];
          cd *du = &tu[(size_t)(tuoff[b] + (int64_t)i * n - (int64_t)i * (i - 1) / 2) * 4];
          for (int j = i; j < n; ++j)
            for (int x = 0; x < 4; ++x) du[4 * (j - i) + x] = blk(X, i, j)[x];
        }
      }
    };
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nth; ++t) th.emplace_back(work);
    for (auto &t : th) t.join();
  }
  IluHost &I = c->ilu;
  I.nboxes = nlb;
  I.colour_ptr = cptr;
  I.max_box = maxb;
  std::vector<int> bl(nlb);
  for (int b = 0; b < nlb; ++b) bl[b] = b;
  I.d_box_start = dev_upload(c, c->leaf_start);
  I.d_box_list = dev_upload(c, bl);
  I.d_lo_ptr = dev_upload(c, lo_ptr);
  I.d_up_ptr = dev_upload(c, up_ptr);
  I.d_lo_col = dev_upload(c, lo_col);
  {
    auto colour_ptrs = [&](const std::vector<int> &ptr, const std::vector<int> &col) {
      std::vector<int> cp((size_t)ne * 9);
      for (int i = 0; i < ne; ++i) {
        int q = ptr[i];
        for (int k = 0; k < 8; ++k) {
          while (q < ptr[i + 1] && bcol[ebox[col[q]]] < k) ++q;
          cp[9 * (size_t)i + k] = q;
        }
        cp[9 * (size_t)i + 8] = ptr[i + 1];
      }
      return cp;
    };
    const std::vector<int> lcp = colour_ptrs(lo_ptr, lo_col), ucp = colour_ptrs(up_ptr, up_col);
    I.d_lo_cptr = dev_upload(c, lcp);
    I.d_up_cptr = dev_upload(c, ucp);
    // pieces of the single-RHS sweep steps: step s < 8 is forward colour s
    // (source colour s - 1), step s >= 8 backward colour 14 - s (source 15 - s)
    const int PIECE = 1024;  // blocks per piece of a box's off-box work
    std::vector<int> pieces, pptr(1, 0);
    size_t maxp = 0;
    for (int step = 0; step < 15; ++step) {
      const bool fwd = step < 8;
      const int colr = fwd ? step : 14 - step, sc = fwd ? colr - 1 : colr + 1;
      const std::vector<int> &cp = fwd ? lcp : ucp;
      size_t here = 0;
      for (int bx = cptr[colr]; bx < cptr[colr + 1]; ++bx) {
        long total = 0;
        if (sc >= 0 && sc < 8)
          for (int i = c->leaf_start[bx]; i < c->leaf_start[bx + 1]; ++i)
            total += cp[9 * (size_t)i + sc + 1] - cp[9 * (size_t)i + sc];
        const int npc = (int)std::max<long>(1, (total + PIECE - 1) / PIECE);
        for (int k = 0; k < npc; ++k) {
          pieces.push_back(bx);
          pieces.push_back((int)(total * k / npc));
          pieces.push_back((int)(total * (k + 1) / npc));
          pieces.push_back(k);
          pieces.push_back(npc);
        }
        here += npc;
      }
      maxp = std::max(maxp, here);
      pptr.push_back((int)(pieces.size() / 5));
    }
    I.piece_ptr = pptr;
    I.d_pieces = dev_upload(c, pieces);
    I.d_piece_count = (int *)dev_alloc(c, (size_t)nlb * sizeof(int));
    SIE_CUDA(cudaMemset(I.d_piece_count, 0, (size_t)nlb * sizeof(int)));
    I.d_piece_scratch = dev_alloc(c, std::max<size_t>(1, maxp) * 2 * std::max(1, maxb) * sizeof(cd));
    I.d_bar = (unsigned *)dev_alloc(c, sizeof(unsigned));
    if (!c->d_err) {
      c->d_err = (int *)dev_alloc(c, sizeof(int));
      SIE_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    }
  }
  I.d_up_col = dev_upload(c, up_col);
  I.d_lo64 = dev_upload(c, lo_val);
  I.d_up64 = dev_upload(c, up_val);
  I.d_tl_off = dev_upload(c, tloff);
  I.d_tu_off = dev_upload(c, tuoff);
  I.d_tl64 = dev_upload(c, tl);
  I.d_tu64 = dev_upload(c, tu);
  auto f32 = [&](const std::vector<cd> &v) {
    std::vector<std::complex<float>> o(v.size());
    for (size_t q = 0; q < v.size(); ++q) o[q] = std::complex<float>((float)v[q].real(), (float)v[q].imag());
    return dev_upload(c, o);
  };
  I.d_lo32 = f32(lo_val);
  I.d_up32 = f32(up_val);
  I.d_tl32 = f32(tl);
  I.d_tu32 = f32(tu);
  I.nblk_off = (int64_t)lo_col.size() + (int64_t)up_col.size();
  I.nblk_inv = (int64_t)(tl.size() + tu.size()) / 4;
  I.ready = true;
}

// ------------------------------------------------------------------ API: fill
static void fill_all(sie_ctx *c, const sie_fill_opts *o) {
  const int ne = c->ne, nt = c->nt;
  int on = o ? o->outer_order : 4;
  c->form = o ? o->formulation : 0;
  SIE_REQUIRE(c->form >= 0 && c->form <= 4, SIE_EINVAL, "sie_fill_nearfield: formulation must be 0..4");
  SIE_REQUIRE(c->form != 4 || c->njunc == 0, SIE_EINVAL,
              "sie_fill_nearfield: ICTF (an interface's mean impedance) is not defined at junction edges");
  SIE_REQUIRE(on >= 2 && on <= 12, SIE_EINVAL, "sie_fill_nearfield: outer_order must be in [2, 12]");
  // geometry tables, internal edge ids
  std::vector<double> tri(22 * (size_t)nt);
  std::vector<int> tri_e(3 * (size_t)nt);
  std::vector<double> tri_sg(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t) {
    double *o2 = &tri[22 * (size_t)t];
    for (int a = 0; a < 3; ++a)
      for (int x = 0; x < 3; ++x) o2[3 * a + x] = c->verts[3 * c->tris[3 * t + a] + x];
    for (int x = 0; x < 3; ++x) o2[9 + x] = c->normal[3 * t + x];
    o2[12] = c->area[t];
    for (int a = 0; a < 3; ++a) {
      int e = c->tri_edge[3 * t + a];
      tri_e[3 * t + a] = e >= 0 ? c->inv[e] : -1;
      tri_sg[3 * t + a] = e >= 0 ? c->tri_sign[3 * t + a] * c->elen[e] / (2.0 * c->area[t]) : 0.0;
      for (int x = 0; x < 3; ++x) o2[13 + 3 * a + x] = c->verts[3 * c->tri_free[3 * t + a] + x];
    }
  }
  c->d_tri = dev_upload(c, tri);
  c->d_tri_e = dev_upload(c, tri_e);
  c->d_tri_sg = dev_upload(c, tri_sg);
  c->d_tri_reg = dev_upload(c, c->tri_reg);
  {
    std::vector<int> t0;
    for (int t = 0; t < nt; ++t)
      if (c->tri_reg[2 * t] == 0 || c->tri_reg[2 * t + 1] == 0) t0.push_back(t);
    c->ntri0 = (int)t0.size();
    if (!t0.empty()) c->d_tri0 = dev_upload(c, t0);
  }
  c->d_row_ptr = dev_upload(c, c->row_ptr);
  c->d_col = dev_upload(c, c->col);
  c->d_perm = dev_upload(c, c->perm);
  c->d_inv = dev_upload(c, c->inv);
  // per basis (internal order): its two triangles in the host medium 0, -1 if it
  // does not bound medium 0 (the excitation tests medium 0's equations only)
  std::vector<int> etri(2 * (size_t)ne, -1);
  for (int p = 0; p < ne; ++p) {
    int e = c->perm[p];
    for (int q = c->emed_ptr[e]; q < c->emed_ptr[e + 1]; ++q)
      if (c->emed[q][0] == 0) {
        etri[2 * p] = c->emed[q][1];
        etri[2 * p + 1] = c->emed[q][2];
      }
  }
  c->d_edge_tris = dev_upload(c, etri);
  // singular outer rule: n x n collapsed Gauss (barycentric b0,b1,b2,w)
  std::vector<double> x, wx, q;
  gauss_legendre(on, x, wx);
  for (int i = 0; i < on; ++i)
    for (int j = 0; j < on; ++j) {
      double u = 0.5 * (x[i] + 1.0), wu = 0.5 * wx[i];
      double v = 0.5 * (x[j] + 1.0), wv = 0.5 * wx[j];
      double xi = u, eta = v * (1.0 - u);
      q.push_back(1.0 - xi - eta);
      q.push_back(xi);
      q.push_back(eta);
      q.push_back(2.0 * wu * wv * (1.0 - u));
    }
  c->nq_sing = on * on;
  c->d_quad = dev_upload(c, q);
  // near matrix
  int64_t nnz = c->row_ptr[ne];
  c->d_near64 = dev_alloc(c, (size_t)nnz * 4 * sizeof(zd));
  c->d_near32 = dev_alloc(c, (size_t)nnz * 4 * sizeof(zf));
  SIE_CUDA(cudaMemsetAsync(c->d_near64, 0, (size_t)nnz * 4 * sizeof(zd), c->stream));
  // triangle pairs per medium: tri p (test) x tri q (source) with some near basis pair
  std::vector<int> tri_int_edges(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) tri_int_edges[3 * t + a] = tri_e[3 * t + a];
  for (int l = 0; l < c->nr; ++l) {
    RegionHost &R = c->reg[l];
    std::vector<int> tl;
    for (int t = 0; t < nt; ++t)
      if (c->tri_reg[2 * t] == l || c->tri_reg[2 * t + 1] == l) tl.push_back(t);
    if (tl.empty()) continue;
    unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::vector<int>> part(nth);
    std::atomic<size_t> next(0);
    auto work = [&](unsigned id) {
      std::vector<int> mark(nt, -1), lst;
      for (;;) {
        size_t ii = next.fetch_add(1);
        if (ii >= tl.size()) break;
        int p = tl[ii];
        lst.clear();
        for (int a = 0; a < 3; ++a) {
          int m = tri_int_edges[3 * p + a];
          if (m < 0) continue;
          for (int e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) {
            int n = c->perm[c->col[e]];
            int ts[2] = {c->tp[n], c->tm[n]};
            for (int s = 0; s < 2; ++s) {
              int qq = ts[s];
              if (mark[qq] == p) continue;
              if (!(c->tri_reg[2 * qq] == l || c->tri_reg[2 * qq + 1] == l)) continue;
              mark[qq] = p;
              lst.push_back(qq);
            }
          }
        }
        std::sort(lst.begin(), lst.end());
        for (int qq : lst) {
          double dx = c->centroid[3 * p] - c->centroid[3 * qq], dy = c->centroid[3 * p + 1] - c->centroid[3 * qq + 1],
                 dz = c->centroid[3 * p + 2] - c->centroid[3 * qq + 2];
          double d = std::sqrt((dx * dx + dy * dy) + dz * dz);
          int sing = d < (c->hmax[p] + c->hmax[qq]) ? 1 : 0;
          part[id].push_back(p);
          part[id].push_back(qq);
          part[id].push_back(sing);
        }
      }
    };
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nth; ++t) th.emplace_back(work, t);
    for (auto &t : th) t.join();
    // singular pairs first (heavier), then regular: keeps warps uniform
    std::vector<int> pairs;
    for (int pass = 1; pass >= 0; --pass)
      for (auto &pv : part)
        for (size_t s = 0; s < pv.size(); s += 3)
          if (pv[s + 2] == pass) pairs.insert(pairs.end(), {pv[s], pv[s + 1], pv[s + 2]});
    R.npairs = (int64_t)pairs.size() / 3;
    R.d_pairs = dev_upload(c, pairs);
    launch_near_fill(c, l);
  }
  launch_identity(c);
  if (c->levels >= 3)
    for (int l = 0; l < c->nr; ++l)
      if (c->reg[l].nb > 0) launch_patterns(c, l);
  launch_to_f32(c, (const double *)c->d_near64, (float *)c->d_near32, nnz * 8);
  if (c->form == 4) {
    // ICTF row weights per basis (internal order): the tangential equations of
    // an interface between media a and b normalised by the mean relative
    // impedance eta~ = (eta~_a + eta~_b) / 2: J-row 1 / eta~, M-row eta~
    std::vector<cd> d((size_t)2 * ne);
    for (int p = 0; p < ne; ++p) {
      const int t = c->tp[c->perm[p]];
      const cd em = 0.5 * (c->etareg[c->tri_reg[2 * t]] + c->etareg[c->tri_reg[2 * t + 1]]);
      d[2 * (size_t)p] = 1.0 / em;
      d[2 * (size_t)p + 1] = em;
    }
    c->rowscale = d;
    c->d_rowscale = dev_upload(c, d);
  }
  SIE_CUDA(cudaStreamSynchronize(c->stream));
  if (!o || o->build_ilu) build_ilu(c);
  c->have_fill = true;
}

extern "C" sie_status sie_fill_nearfield(sie_ctx *c, const sie_fill_opts *o) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_tree, SIE_ESTATE, "sie_fill_nearfield: call mlfmm_setup first");
    SIE_REQUIRE(!c->have_fill, SIE_ESTATE, "sie_fill_nearfield: already filled");
    fill_all(c, o);
  });
}

// ------------------------------------------------------------------ API: operator
extern "C" sie_status sie_matvec_parts(sie_ctx *c, const void *x, void *y, int64_t nrhs, sie_prec prec,
                                       int32_t parts) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "matvec: call sie_fill_nearfield first");
    SIE_REQUIRE(x && y && x != y && nrhs >= 1 && nrhs <= 4096, SIE_EINVAL, "matvec: bad buffers or nrhs");
    SIE_REQUIRE(prec == SIE_PREC_FP64 || prec == SIE_PREC_MIXED || prec == SIE_PREC_NEAR64, SIE_EINVAL,
                "matvec: bad precision");
    SIE_REQUIRE(parts >= 1 && parts <= 3, SIE_EINVAL, "matvec: parts must be 1, 2 or 3");
    ensure_work(c, nrhs);
    op_permute_in(c, (const zd *)x, (zd *)c->d_xi, (int)nrhs);
    apply_matvec(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs, prec, parts);
    op_permute_out(c, (const zd *)c->d_yi, (zd *)y, (int)nrhs);
  });
}

extern "C" sie_status mlfmm_matvec(sie_ctx *c, const void *x, void *y, int64_t nrhs, sie_prec prec) {
  return sie_matvec_parts(c, x, y, nrhs, prec, 3);
}

extern "C" sie_status ilu_apply(sie_ctx *c, const void *r, void *z, int64_t nrhs, sie_prec prec) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_fill && c->ilu.ready, SIE_ESTATE, "ilu_apply: no ILU factors (fill with build_ilu)");
    SIE_REQUIRE(r && z && r != z && nrhs >= 1 && nrhs <= 4096, SIE_EINVAL, "ilu_apply: bad buffers or nrhs");
    SIE_REQUIRE(prec == SIE_PREC_FP64 || prec == SIE_PREC_MIXED, SIE_EINVAL, "ilu_apply: bad precision");
    ensure_work(c, nrhs);
    op_permute_in(c, (const zd *)r, (zd *)c->d_xi, (int)nrhs);
    apply_ilu(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs, prec);
    op_permute_out(c, (const zd *)c->d_yi, (zd *)z, (int)nrhs);
  });
}

extern "C" sie_status sie_plane_wave_rhs(sie_ctx *c, const double *inc, int64_t nrhs, void *b) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "sie_plane_wave_rhs: call sie_fill_nearfield first");
    SIE_REQUIRE(inc && b && nrhs >= 1 && nrhs <= 4096, SIE_EINVAL, "sie_plane_wave_rhs: bad arguments");
    ensure_work(c, nrhs);
    double *d_inc = (double *)stage(c, (size_t)nrhs * 4 * sizeof(double));
    SIE_CUDA(cudaMemcpyAsync(d_inc, inc, (size_t)nrhs * 4 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_rhs(c, d_inc, (int)nrhs, (zd *)c->d_xi);
    op_permute_out(c, (const zd *)c->d_xi, (zd *)b, (int)nrhs);
    SIE_CUDA(cudaStreamSynchronize(c->stream));
  });
}

extern "C" sie_status gmres_solve(sie_ctx *c, const void *b, void *x, int64_t nrhs, const sie_solve_opts *o,
                                  sie_solve_stats *st) {
  sie_status rc = SIE_OK;
  sie_status g = guard(c, [&] {
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "gmres_solve: call sie_fill_nearfield first");
    SIE_REQUIRE(b && x && o && st && nrhs >= 1 && nrhs <= 4096, SIE_EINVAL, "gmres_solve: bad arguments");
    SIE_REQUIRE(o->restart >= 1 && o->restart <= 500 && o->max_iters >= 1 && o->tol > 0, SIE_EINVAL,
                "gmres_solve: bad options");
    SIE_REQUIRE(o->precond >= 0 && o->precond <= 2, SIE_EINVAL, "gmres_solve: precond must be 0, 1 or 2");
    SIE_REQUIRE(o->method >= 0 && o->method <= 2, SIE_EINVAL, "gmres_solve: method must be 0, 1 or 2");
    SIE_REQUIRE(o->prec == SIE_PREC_FP64 || o->prec == SIE_PREC_MIXED, SIE_EINVAL, "gmres_solve: prec must be 0 or 1");
    SIE_REQUIRE(o->residual_far_fp64 == 0 || o->residual_far_fp64 == 1, SIE_EINVAL,
                "gmres_solve: residual_far_fp64 must be 0 or 1");
    SIE_REQUIRE(o->method == 0 || o->precond <= 1, SIE_EINVAL,
                "gmres_solve: the learned correction needs FGMRES (a variable preconditioner)");
    SIE_REQUIRE(o->precond == 0 || c->ilu.ready, SIE_ESTATE, "gmres_solve: ILU requested but not built");
    SIE_REQUIRE(o->precond != 2 || nn_trained(c), SIE_ESTATE, "gmres_solve: learned preconditioner not trained");
    rc = run_gmres(c, (const zd *)b, (zd *)x, (int)nrhs, o, st);
  });
  return g != SIE_OK ? g : rc;
}

extern "C" sie_status rcs_farfield_prec(sie_ctx *c, const void *x, int64_t nrhs, const double *obs, int64_t nobs,
                                        int32_t prec, double *rcs) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "rcs_farfield: call sie_fill_nearfield first");
    SIE_REQUIRE(x && obs && rcs && nrhs >= 1 && nobs >= 1 && nrhs <= 4096 && nobs <= 1000000, SIE_EINVAL,
                "rcs_farfield: bad arguments");
    SIE_REQUIRE(prec == SIE_PREC_FP64 || prec == SIE_PREC_MIXED, SIE_EINVAL, "rcs_farfield: prec must be 0 or 1");
    ensure_work(c, nrhs);
    op_permute_in(c, (const zd *)x, (zd *)c->d_xi, (int)nrhs);
    size_t ob = ((size_t)nobs * 2 * sizeof(double) + 255) / 256 * 256;
    double *d_obs = (double *)stage(c, ob + (size_t)nrhs * nobs * 2 * sizeof(double));
    double *d_out = (double *)((char *)d_obs + ob);
    SIE_CUDA(cudaMemcpyAsync(d_obs, obs, (size_t)nobs * 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_farfield(c, (const zd *)c->d_xi, (int)nrhs, d_obs, (int)nobs, d_out, (sie_prec)prec);
    SIE_CUDA(cudaMemcpyAsync(rcs, d_out, (size_t)nrhs * nobs * 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SIE_CUDA(cudaStreamSynchronize(c->stream));
  });
}

extern "C" sie_status rcs_farfield(sie_ctx *c, const void *x, int64_t nrhs, const double *obs, int64_t nobs,
                                   double *rcs) {
  return rcs_farfield_prec(c, x, nrhs, obs, nobs, SIE_PREC_FP64, rcs);
}

extern "C" sie_status sie_near_export(sie_ctx *c, int32_t *rows, int32_t *cols, double *vals, int64_t *nnzb) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "sie_near_export: call sie_fill_nearfield first");
    SIE_REQUIRE(nnzb, SIE_EINVAL, "sie_near_export: null nnzb");
    int64_t nnz = c->row_ptr[c->ne];
    *nnzb = nnz;
    if (!rows) return;
    SIE_REQUIRE(cols && vals, SIE_EINVAL, "sie_near_export: null cols/vals");
    SIE_CUDA(cudaStreamSynchronize(c->stream));
    SIE_CUDA(cudaMemcpy(vals, c->d_near64, (size_t)nnz * 8 * sizeof(double), cudaMemcpyDeviceToHost));
    for (int p = 0; p < c->ne; ++p)
      for (int e = c->row_ptr[p]; e < c->row_ptr[p + 1]; ++e) {
        rows[e] = c->perm[p];
        cols[e] = c->perm[c->col[e]];
      }
  });
}

// Mean device milliseconds of one launch of a stage of the hot path (after one
// warm-up launch), CUDA events on the context's stream.
static double time_stage(sie_ctx *c, int stage, int64_t nrhs, int prec, int reps) {
  {
    ensure_work(c, nrhs);
    size_t n = (size_t)nrhs * c->ne * 2;
    SIE_CUDA(cudaMemsetAsync(c->d_xi, 0, n * sizeof(zd), c->stream));
    SIE_CUDA(cudaMemsetAsync(c->d_xf, 0, n * sizeof(zf), c->stream));
    cudaEvent_t e0, e1;
    SIE_CUDA(cudaEventCreate(&e0));
    SIE_CUDA(cudaEventCreate(&e1));
    auto run = [&]() {
      bool f64 = prec == SIE_PREC_FP64;
      switch (stage) {
        case 0:
          if (f64) op_near<double>(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs, false);
          else op_near<float>(c, (const zf *)c->d_xf, (zf *)c->d_yf, (int)nrhs, false);
          break;
        case 1:
          if (f64) op_far<double>(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs);
          else op_far<float>(c, (const zf *)c->d_xf, (zf *)c->d_yf, (int)nrhs);
          break;
        case 2:
          if (f64) op_ilu<double>(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs);
          else op_ilu<float>(c, (const zf *)c->d_xf, (zf *)c->d_yf, (int)nrhs);
          break;
        default:
          if (prec == SIE_PREC_NEAR64) {
            apply_matvec(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs, SIE_PREC_NEAR64, 3);
          } else if (f64) {
            op_near<double>(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs, false);
            op_far<double>(c, (const zd *)c->d_xi, (zd *)c->d_yi, (int)nrhs);
          } else {
            op_near<float>(c, (const zf *)c->d_xf, (zf *)c->d_yf, (int)nrhs, false);
            op_far<float>(c, (const zf *)c->d_xf, (zf *)c->d_yf, (int)nrhs);
          }
      }
    };
    run();  // warm-up
    SIE_CUDA(cudaEventRecord(e0, c->stream));
    for (int i = 0; i < reps; ++i) run();
    SIE_CUDA(cudaEventRecord(e1, c->stream));
    SIE_CUDA(cudaEventSynchronize(e1));
    float t = 0;
    SIE_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)t / reps;
  }
}

extern "C" sie_status sie_stage_timing(sie_ctx *c, int32_t stage, int64_t nrhs, int32_t prec, int32_t reps,
                                       double *ms) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "sie_stage_timing: call sie_fill_nearfield first");
    SIE_REQUIRE(ms && stage >= 0 && stage <= 3 && nrhs >= 1 && nrhs <= 4096 && reps >= 1, SIE_EINVAL,
                "sie_stage_timing: bad arguments");
    SIE_REQUIRE(stage != 2 || c->ilu.ready, SIE_ESTATE, "sie_stage_timing: no ILU factors");
    SIE_REQUIRE(prec == SIE_PREC_FP64 || prec == SIE_PREC_MIXED || (prec == SIE_PREC_NEAR64 && stage == 3),
                SIE_EINVAL, "sie_stage_timing: prec 0 or 1 (2 for the whole product only)");
    *ms = time_stage(c, stage, nrhs, prec, reps);
  });
}

// Autotuner of the block-RHS tile shapes: for each tunable parameter in turn
// (coordinate descent), time the stage it belongs to for each candidate value
// with the others held, keep the fastest.  FP32 (mixed-form) kernels.
extern "C" sie_status sie_autotune(sie_ctx *c, int64_t nrhs, int32_t reps, int64_t *choice, double *ms) {
  return guard(c, [&] {
    SIE_REQUIRE(c->have_fill, SIE_ESTATE, "sie_autotune: call sie_fill_nearfield first");
    SIE_REQUIRE(choice && nrhs >= 2 && nrhs <= 4096 && reps >= 1, SIE_EINVAL, "sie_autotune: bad arguments");
    const int R = (int)nrhs;
    graphs_free(c);
    auto best_of = [&](int stage, int *param, std::initializer_list<int> cands) {
      double tbest = 1e300;
      int vbest = *param;
      for (int v : cands) {
        *param = v;
        const double t = time_stage(c, stage, R, SIE_PREC_MIXED, reps);
        if (t < tbest) {
          tbest = t;
          vbest = v;
        }
      }
      *param = vbest;
      return tbest;
    };
    double t_near = best_of(0, &c->tune_near_rb, {4, 8, 16});
    double t_ilu = c->ilu.ready ? best_of(2, &c->tune_ilu_rb, {4, 8, 16}) : 0.0;
    // far field: aggregation (0 SIMT, else tensor cores with that many right-hand
    // sides per pass), receive passes, M2L form
    int agg = 0;
    {
      std::vector<int> cands{0};
      for (int rb : {16, 32, 64})
        if (R >= 16 && rb <= std::max(16, R)) cands.push_back(rb);
      double tb = 1e300;
      for (int v : cands) {
        c->agg_tc_min_rhs = v ? 2 : 0;
        c->agg_tc_rb = v;
        const double t = time_stage(c, 1, R, SIE_PREC_MIXED, reps);
        if (t < tb) {
          tb = t;
          agg = v;
        }
      }
      c->agg_tc_min_rhs = agg ? 2 : 0;
      c->agg_tc_rb = agg;
    }
    best_of(1, &c->tune_rec_rb, {1, 2, 4});
    if (R >= 16) best_of(1, &c->rec_tc_rb, {0, 16, 32, 64});
    double t_far = best_of(1, &c->tune_m2l, {0, 1, 2});
    choice[0] = c->tune_near_rb;
    choice[1] = c->tune_ilu_rb;
    choice[2] = agg;
    choice[3] = c->tune_rec_rb;
    choice[4] = c->tune_m2l;
    choice[5] = c->rec_tc_rb;
    if (ms) {
      ms[0] = t_near;
      ms[1] = t_ilu;
      ms[2] = t_far;
    }
    graphs_free(c);
  });
}

extern "C" sie_status sie_device_status(sie_ctx *c) {
  return guard(c, [&] { check_device_error(c); });
}

extern "C" sie_status sie_set_param(sie_ctx *c, int32_t key, int64_t value) {
  return guard(c, [&] {
    switch (key) {
      case 0:
        SIE_REQUIRE(value >= 0 && value <= (1ll << 30), SIE_EINVAL, "sie_set_param: wait limit out of range");
        c->wait_limit = (int)value;
        graphs_free(c);  // captured steps hold the limit as a launch argument
        break;
      case 1:
        SIE_REQUIRE(value == 0 || value == 1, SIE_EINVAL, "sie_set_param: ILU schedule must be 0 or 1");
        c->ilu_schedule = (int)value;
        graphs_free(c);  // captured steps hold the other schedule's launches
        break;
      case 2:
        SIE_REQUIRE(value >= 0 && value <= 4096, SIE_EINVAL, "sie_set_param: tensor-core aggregation threshold out of range");
        c->agg_tc_min_rhs = (int)value;
        graphs_free(c);
        break;
      case 3:
        SIE_REQUIRE(value == 0 || value == 16 || value == 32 || value == 64, SIE_EINVAL,
                    "sie_set_param: tensor-core aggregation block must be 0, 16, 32 or 64");
        c->agg_tc_rb = (int)value;
        graphs_free(c);
        break;
      case 4:
      case 5:
        SIE_REQUIRE(value == 0 || value == 4 || value == 8 || value == 16, SIE_EINVAL,
                    "sie_set_param: block size must be 0, 4, 8 or 16");
        (key == 4 ? c->tune_near_rb : c->tune_ilu_rb) = (int)value;
        graphs_free(c);
        break;
      case 6:
        SIE_REQUIRE(value == 0 || value == 1 || value == 2 || value == 4, SIE_EINVAL,
                    "sie_set_param: receive block must be 0, 1, 2 or 4");
        c->tune_rec_rb = (int)value;
        graphs_free(c);
        break;
      case 7:
        SIE_REQUIRE(value >= -1 && value <= 2, SIE_EINVAL, "sie_set_param: M2L form must be -1, 0, 1 or 2");
        c->tune_m2l = (int)value;
        graphs_free(c);
        break;
      case 8:
        SIE_REQUIRE(value == -1 || value == 0 || value == 16 || value == 32 || value == 64, SIE_EINVAL,
                    "sie_set_param: tensor-core receive block must be -1, 0, 16, 32 or 64");
        c->rec_tc_rb = (int)value;
        graphs_free(c);
        break;
      case 9:
        SIE_REQUIRE(value == 0 || value == 1, SIE_EINVAL, "sie_set_param: learned-preconditioner layers must be 0 or 1");
        c->nn_tc = (int)value;
        graphs_free(c);
        break;
      case 10:
        SIE_REQUIRE(value >= -1 && value <= 1, SIE_EINVAL, "sie_set_param: interpolation split must be -1, 0 or 1");
        c->tune_interp_split = (int)value;
        graphs_free(c);
        break;
      default:
        throw SieError{SIE_EINVAL, "sie_set_param: unknown key"};
    }
  });
}

extern "C" sie_status sie_query(const sie_ctx *c, int32_t key, int64_t *v) {
  if (!c || !v) return SIE_EINVAL;
  switch (key) {
    case 0: *v = c->ne; return SIE_OK;
    case 1: *v = c->have_tree ? c->row_ptr[c->ne] : 0; return SIE_OK;
    case 2: *v = c->levels; return SIE_OK;
    case 3: *v = c->nr; return SIE_OK;
    case 4: *v = c->have_tree ? (int64_t)c->leaf_start.size() - 1 : 0; return SIE_OK;
    case 5: *v = c->have_tree ? (int64_t)c->row_ptr[c->ne] * 64 : 0; return SIE_OK;
    case 6: {
      int64_t s = 0;
      for (auto &R : c->reg)
        if (R.nb > 0 && c->levels > 0) s += (int64_t)R.nb * 4 * R.lev[c->levels - 1].K * 16;
      *v = s;
      return SIE_OK;
    }
    case 7: *v = c->dev_bytes; return SIE_OK;
    case 8: *v = c->launches; return SIE_OK;
    case 9:  // algorithmic bytes of one single-RHS FP32 ILU(0) apply
      *v = c->ilu.ready ? c->ilu.nblk_off * (32 + 4) + c->ilu.nblk_inv * 32 + (int64_t)c->ne * (2 * 9 * 4 + 2 * 16) : 0;
      return SIE_OK;
    case 10: *v = graphs_state(c); return SIE_OK;
    default:
      if (key >= 100 && key < 100 + 16 * 64) {
        int l = (key - 100) / 16, j = (key - 100) % 16;
        if (l < (int)c->reg.size() && j < (int)c->reg[l].lev.size()) {
          *v = c->reg[l].lev[j].K;
          return SIE_OK;
        }
      }
      return SIE_EINVAL;
  }
}
