// Setup-time kernels in FP64: near-field Galerkin fill with singularity
// extraction (Eqs. 23-26, identity terms of Eqs. 8-11), leaf radiation and
// receive patterns for the MLFMM, tested plane-wave excitation (Eqs. 20-21,
// Eq. 30) and far field / RCS (Eqs. 27-29).
#include <cmath>

#include <algorithm>

#include "common.h"

namespace {

// Radon's 7-point degree-5 rule on a triangle (barycentric, weights sum to 1).
__constant__ double c_rb[7][3];
__constant__ double c_rw[7];
bool g_rule_ready = false;

void upload_radon() {
  if (g_rule_ready) return;
  const double s = std::sqrt(15.0);
  const double a1 = (6.0 - s) / 21.0, a2 = (6.0 + s) / 21.0;
  const double w1 = (155.0 - s) / 1200.0, w2 = (155.0 + s) / 1200.0;
  double b[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                    {1 - 2 * a1, a1, a1}, {a1, 1 - 2 * a1, a1}, {a1, a1, 1 - 2 * a1},
                    {1 - 2 * a2, a2, a2}, {a2, 1 - 2 * a2, a2}, {a2, a2, 1 - 2 * a2}};
  double w[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
  SIE_CUDA(cudaMemcpyToSymbol(c_rb, b, sizeof(b)));
  SIE_CUDA(cudaMemcpyToSymbol(c_rw, w, sizeof(w)));
  g_rule_ready = true;
}

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 v3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(V3 a) { return sqrt(dot(a, a)); }

// complex 3-vector
struct C3 {
  zd x, y, z;
};
__device__ __forceinline__ zd cdot(V3 a, const C3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ C3 ccross(const C3 &a, V3 b) {  // a x b, a complex, b real
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

struct Tri {
  V3 v[3], n, fr[3];
  double A;
  int e[3];
  double c[3];  // sigma * l / (2A)
};
__device__ __forceinline__ void load_tri(const double *tri, const int *te, const double *tsg, int t, Tri &T) {
  const double *o = tri + 22 * (size_t)t;
  for (int a = 0; a < 3; ++a) T.v[a] = v3(o[3 * a], o[3 * a + 1], o[3 * a + 2]);
  T.n = v3(o[9], o[10], o[11]);
  T.A = o[12];
  for (int a = 0; a < 3; ++a) {
    T.fr[a] = v3(o[13 + 3 * a], o[14 + 3 * a], o[15 + 3 * a]);
    T.e[a] = te[3 * t + a];
    T.c[a] = tsg[3 * t + a];
  }
}
__device__ __forceinline__ V3 bary(const Tri &T, double b0, double b1, double b2) {
  return b0 * T.v[0] + b1 * T.v[1] + b2 * T.v[2];
}

// exp(-j k R) for complex k = kr + j ki
__device__ __forceinline__ zd expmjkR(zd k, double R) {
  double mag = exp(k.im * R);
  double s, c;
  sincos(k.re * R, &s, &c);
  return zd(mag * c, -mag * s);
}

// Closed-form integrals of 1/R, (rho' - rho)/R and grad_r(1/R) over a flat
// triangle (Wilton et al. 1984; Graglia 1993), written from the geometry.
__device__ void tri_potentials(V3 r, const Tri &T, double &I1, V3 &Irho, V3 &Igr, V3 &rho) {
  V3 n = cross(T.v[1] - T.v[0], T.v[2] - T.v[0]);
  n = (1.0 / norm(n)) * n;
  double w = dot(r - T.v[0], n);
  double scale = norm(T.v[1] - T.v[0]);
  if (fabs(w) < 1e-12 * scale) w = 0.0;
  rho = r - w * n;
  double aw = fabs(w);
  I1 = 0.0;
  Irho = v3(0, 0, 0);
  Igr = v3(0, 0, 0);
  double sb = 0.0;
  for (int s = 0; s < 3; ++s) {
    V3 a = T.v[s], b = T.v[(s + 1) % 3];
    V3 el = b - a;
    V3 l = (1.0 / norm(el)) * el;
    V3 u = cross(l, n);
    double sm = dot(a - rho, l), sp = dot(b - rho, l), t0 = dot(a - rho, u);
    double R02 = t0 * t0 + w * w;
    double Rp = norm(r - b), Rm = norm(r - a);
    double f;
    if (sp < 0 && sm < 0) {
      f = log((Rm - sm) / (Rp - sp));
    } else {
      double Ap = sp >= 0 ? Rp + sp : R02 / (Rp - sp);
      double Am = sm >= 0 ? Rm + sm : R02 / (Rm - sm);
      f = log(Ap / Am);
    }
    double beta = atan2(t0 * sp, R02 + aw * Rp) - atan2(t0 * sm, R02 + aw * Rm);
    I1 += t0 * f;
    Irho = Irho + (0.5 * (R02 * f + sp * Rp - sm * Rm)) * u;
    Igr = Igr - f * u;
    sb += beta;
  }
  I1 -= aw * sb;
  double sg = (w > 0) - (w < 0);
  Igr = Igr - (sg * sb) * n;
}

// One near triangle pair of medium `l`: Galerkin values of L, K, n x L, n x K
// for the 3x3 local bases, combined into JMCFIE blocks and added to the
// block-sparse near matrix.
__global__ void k_near_fill(const int *pairs, int64_t npairs, const double *tri, const int *te, const double *tsg,
                            const int *treg, int region, zd k, zd eta, const double *quad, int nq,
                            const int *row_ptr, const int *col, double *near, zd aTJ, zd aNJ, zd aTM, zd aNM) {
  int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= npairs) return;
  int p = pairs[3 * id], q = pairs[3 * id + 1], sing = pairs[3 * id + 2];
  Tri P, Q;
  load_tri(tri, te, tsg, p, P);
  load_tri(tri, te, tsg, q, Q);
  const zd jk = zd(-k.im, k.re);                  // j k
  const double kk2 = k.re * k.re + k.im * k.im;
  const zd joverk = zd(k.im / kk2, k.re / kk2);   // j / k
  zd L[3][3], K[3][3], NL[3][3], NK[3][3], SG;
  const int na = sing ? nq : 7;
  const double inv4pi = 1.0 / (4.0 * M_PI);
  for (int a = 0; a < na; ++a) {
    double b0, b1, b2, wa;
    if (sing) {
      b0 = quad[4 * a]; b1 = quad[4 * a + 1]; b2 = quad[4 * a + 2]; wa = quad[4 * a + 3];
    } else {
      b0 = c_rb[a][0]; b1 = c_rb[a][1]; b2 = c_rb[a][2]; wa = c_rw[a];
    }
    V3 r = bary(P, b0, b1, b2);
    double W = P.A * wa;
    zd IG;
    C3 IGr = {zd(), zd(), zd()}, IgG = {zd(), zd(), zd()};
    if (!sing) {
      for (int b = 0; b < 7; ++b) {
        V3 rq = bary(Q, c_rb[b][0], c_rb[b][1], c_rb[b][2]);
        double Wq = Q.A * c_rw[b];
        V3 D = r - rq;
        double R = norm(D);
        zd e = expmjkR(k, R);
        zd G = (Wq * inv4pi / R) * e;
        IG += G;
        IGr.x += rq.x * G; IGr.y += rq.y * G; IGr.z += rq.z * G;
        zd g = (-Wq * inv4pi / (R * R * R)) * ((zd(1.0, 0.0) + R * jk) * e);
        IgG.x += D.x * g; IgG.y += D.y * g; IgG.z += D.z * g;
      }
    } else {
      double I1;
      V3 Irho, Igr, rho;
      tri_potentials(r, Q, I1, Irho, Igr, rho);
      zd remS;
      C3 remR = {zd(), zd(), zd()}, remG = {zd(), zd(), zd()};
      for (int b = 0; b < 7; ++b) {
        V3 rq = bary(Q, c_rb[b][0], c_rb[b][1], c_rb[b][2]);
        double Wq = Q.A * c_rw[b];
        V3 D = r - rq;
        double R = norm(D);
        zd rm, gr;
        if (R < 1e-14) {
          rm = zd(k.im, -k.re);  // -j k
          gr = zd();
        } else {
          zd e = expmjkR(k, R);
          rm = (1.0 / R) * (e - zd(1.0, 0.0));
          gr = (1.0 / (R * R * R)) * (zd(1.0, 0.0) - (zd(1.0, 0.0) + R * jk) * e);
        }
        rm = Wq * rm;
        gr = Wq * gr;
        remS += rm;
        remR.x += rq.x * rm; remR.y += rq.y * rm; remR.z += rq.z * rm;
        remG.x += D.x * gr; remG.y += D.y * gr; remG.z += D.z * gr;
      }
      IG = inv4pi * (zd(I1, 0.0) + remS);
      IGr.x = inv4pi * (zd(Irho.x + rho.x * I1, 0.0) + remR.x);
      IGr.y = inv4pi * (zd(Irho.y + rho.y * I1, 0.0) + remR.y);
      IGr.z = inv4pi * (zd(Irho.z + rho.z * I1, 0.0) + remR.z);
      IgG.x = inv4pi * (zd(Igr.x, 0.0) + remG.x);
      IgG.y = inv4pi * (zd(Igr.y, 0.0) + remG.y);
      IgG.z = inv4pi * (zd(Igr.z, 0.0) + remG.z);
    }
    SG += W * IG;
    V3 Fm[3], Fmn[3];
    for (int i = 0; i < 3; ++i) {
      Fm[i] = P.c[i] * (r - P.fr[i]);
      Fmn[i] = cross(Fm[i], P.n);
    }
    for (int j = 0; j < 3; ++j) {
      double cj = Q.c[j];
      C3 Fn = {cj * (IGr.x - Q.fr[j].x * IG), cj * (IGr.y - Q.fr[j].y * IG), cj * (IGr.z - Q.fr[j].z * IG)};
      C3 Cr = ccross(IgG, r - Q.fr[j]);
      Cr.x = cj * Cr.x; Cr.y = cj * Cr.y; Cr.z = cj * Cr.z;
      double dj = 2.0 * cj;
      for (int i = 0; i < 3; ++i) {
        L[i][j] += W * (jk * cdot(Fm[i], Fn));
        K[i][j] += W * cdot(Fm[i], Cr);
        NL[i][j] += W * (jk * cdot(Fmn[i], Fn) + (dj * joverk) * cdot(Fmn[i], IgG));
        NK[i][j] += W * cdot(Fmn[i], Cr);
      }
    }
  }
  const double sm = treg[2 * p] == region ? 1.0 : -1.0;
  const double sn = treg[2 * q] == region ? 1.0 : -1.0;
  const double ss = sm * sn;
  const zd ieta = zd(eta.re, -eta.im) * (1.0 / (eta.re * eta.re + eta.im * eta.im));
  for (int i = 0; i < 3; ++i) {
    int m = P.e[i];
    if (m < 0) continue;
    int lo = row_ptr[m], hi = row_ptr[m + 1];
    for (int j = 0; j < 3; ++j) {
      int nn = Q.e[j];
      if (nn < 0) continue;
      int a = lo, b = hi;  // binary search for column nn
      while (a < b) {
        int mid = (a + b) >> 1;
        if (col[mid] < nn) a = mid + 1; else b = mid;
      }
      if (a >= hi || col[a] != nn) continue;  // far pair: carried by the MLFMM
      zd Lij = L[i][j] - ((2.0 * P.c[i]) * (2.0 * Q.c[j])) * (joverk * SG);
      // J-row = sum_l s_l [aTJ T-EFIE_l / eta_l - aNJ N-MFIE_l],
      // M-row = sum_l s_l [aNM N-EFIE_l - aTM eta_l T-MFIE_l]
      const zd tl = ss * Lij, nk = -(sn * NK[i][j]), tk = ss * K[i][j], nl = sn * NL[i][j];
      zd jj = aTJ * tl + aNJ * nk;
      zd jm = (aTJ * tk + aNJ * nl) * ieta;
      zd mj = -((aTM * tk + aNM * nl) * eta);
      zd mm = aTM * tl + aNM * nk;
      double *o = near + 8 * (size_t)a;
      atomicAdd(o + 0, jj.re); atomicAdd(o + 1, jj.im);
      atomicAdd(o + 2, jm.re); atomicAdd(o + 3, jm.im);
      atomicAdd(o + 4, mj.re); atomicAdd(o + 5, mj.im);
      atomicAdd(o + 6, mm.re); atomicAdd(o + 7, mm.im);
    }
  }
}

// Identity (Gram) terms of both media of each triangle: +1/2 <t, b> per
// side on the J and M rows (normal parts, weights aNJ / aNM), +-1/2 <t, n x b>
// weighted by eta~ per side (tangential parts, weights aTJ / aTM).
// w: per medium (aTJ, aNJ, aTM, aNM).
__global__ void k_identity(int nt, const double *tri, const int *te, const double *tsg, const int *treg,
                           const zd *etas, const zd *w, const int *row_ptr, const int *col, double *near,
                           int *err) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  Tri P;
  load_tri(tri, te, tsg, t, P);
  double Gm[3][3] = {}, Gx[3][3] = {};
  for (int a = 0; a < 7; ++a) {
    V3 r = bary(P, c_rb[a][0], c_rb[a][1], c_rb[a][2]);
    double W = P.A * c_rw[a];
    V3 F[3];
    for (int i = 0; i < 3; ++i) F[i] = P.c[i] * (r - P.fr[i]);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Gm[i][j] += W * dot(F[i], F[j]);
        Gx[i][j] += W * dot(F[i], cross(P.n, F[j]));
      }
  }
  const int lp = treg[2 * t], lm = treg[2 * t + 1];
  zd ep = etas[lp], em = etas[lm];
  const zd *wp = w + 4 * lp, *wm = w + 4 * lm;
  auto inv = [](zd z) { return zd(z.re, -z.im) * (1.0 / (z.re * z.re + z.im * z.im)); };
  zd cjm = 0.5 * (wp[0] * inv(ep) - wm[0] * inv(em));
  zd cmj = -0.5 * (wp[2] * ep - wm[2] * em);
  zd cjj = 0.5 * (wp[1] + wm[1]), cmm = 0.5 * (wp[3] + wm[3]);
  for (int i = 0; i < 3; ++i) {
    int m = P.e[i];
    if (m < 0) continue;
    for (int j = 0; j < 3; ++j) {
      int nn = P.e[j];
      if (nn < 0) continue;
      int a = row_ptr[m], b = row_ptr[m + 1], hi = b;
      while (a < b) {
        int mid = (a + b) >> 1;
        if (col[mid] < nn) a = mid + 1; else b = mid;
      }
      if (a >= hi || col[a] != nn) {
        atomicExch(err, 1);
        continue;
      }
      double *o = near + 8 * (size_t)a;
      zd jm = Gx[i][j] * cjm, mj = Gx[i][j] * cmj, jj = Gm[i][j] * cjj, mm = Gm[i][j] * cmm;
      atomicAdd(o + 0, jj.re); atomicAdd(o + 1, jj.im);
      atomicAdd(o + 2, jm.re); atomicAdd(o + 3, jm.im);
      atomicAdd(o + 4, mj.re); atomicAdd(o + 5, mj.im);
      atomicAdd(o + 6, mm.re); atomicAdd(o + 7, mm.im);
    }
  }
}

// Leaf patterns of medium l at direction k:
//   V_i(k)  = int b_i e^{+j k khat.(r - c_b)}          (radiation, theta/phi)
//   RN_i(k) = int (t_i x n) e^{-j k khat.(r - c_b)}     (receive of n x operators)
// over the basis's two triangles in this medium (ptri), each triangle's piece
// of V weighted by psg (1 for an ordinary edge, whose medium sign is applied
// by the aggregation and the receive; the side sign s_l(T) at a junction edge,
// whose two triangles in this medium lie on different surfaces).  RN needs no
// such sign: the piece and the medium's normal change sign together.
__global__ void k_patterns(int nb, int K, const int *basis_p, const int *basis_box, const double *centre,
                           const int *ptri, const double *psg, const double *tri, const int *te, const double *tsg,
                           const double *dirs, zd k, zd *V, zd *RN) {
  int kk = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (kk >= K || i >= nb) return;
  int p = basis_p[i];
  const double *cb = centre + 3 * basis_box[i];
  V3 c = v3(cb[0], cb[1], cb[2]);
  const double *d = dirs + 9 * kk;
  V3 kh = v3(d[0], d[1], d[2]), th = v3(d[3], d[4], d[5]), ph = v3(d[6], d[7], d[8]);
  zd vt, vp, rt, rp;
  for (int s = 0; s < 2; ++s) {
    int t = ptri[2 * i + s];
    const double sv = psg[2 * i + s];
    Tri T;
    load_tri(tri, te, tsg, t, T);
    int li = 0;
    for (int a = 0; a < 3; ++a)
      if (T.e[a] == p) li = a;
    for (int a = 0; a < 7; ++a) {
      V3 r = bary(T, c_rb[a][0], c_rb[a][1], c_rb[a][2]);
      double W = T.A * c_rw[a];
      V3 fn = cross(T.c[li] * (r - T.fr[li]), T.n);
      V3 f = (sv * T.c[li]) * (r - T.fr[li]);
      double x = dot(kh, r - c);
      // e^{+jkx} = e^{-k_i x} (cos k_r x + j sin k_r x)
      double s1, c1;
      sincos(k.re * x, &s1, &c1);
      double gp = exp(-k.im * x), gm = exp(k.im * x);
      zd ep(gp * c1, gp * s1), em(gm * c1, -gm * s1);
      vt += (W * dot(f, th)) * ep;
      vp += (W * dot(f, ph)) * ep;
      rt += (W * dot(fn, th)) * em;
      rp += (W * dot(fn, ph)) * em;
    }
  }
  V[((size_t)i * 2 + 0) * K + kk] = vt;
  V[((size_t)i * 2 + 1) * K + kk] = vp;
  RN[((size_t)i * 2 + 0) * K + kk] = rt;
  RN[((size_t)i * 2 + 1) * K + kk] = rp;
}

// Combined receive pattern of basis i in medium l, so that the leaf receive
// reads one pattern per basis instead of two:
//   P_t(k) = s_i V_t(-k) + RN_p(k),   P_p(k) = -s_i V_p(-k) - RN_t(k),
// V(-k) taken at the antipodal sample (theta row L - it, phi column + pi),
// where the theta unit vector is the same and the phi unit vector reversed.
// Written over RN in place (each thread reads only its own RN entries).
// With the formulation's tangential and normal weights aT, aN (equal on
// both rows; PMCHWT's per-row impedance factors are applied at the receive).
__global__ void k_receive_fold(int nb, int K, int L, const int *sign, const zd *V, zd *RN, double aT, double aN) {
  const int kk = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (kk >= K || i >= nb) return;
  const int nph = 2 * L + 2, it = kk / nph, jp = kk - it * nph;
  const int ka = (L - it) * nph + (jp + L + 1) % nph;
  const double s = aT * (double)sign[i];
  const zd *Vi = V + (size_t)i * 2 * K;
  zd *Ri = RN + (size_t)i * 2 * K;
  const zd rt = Ri[kk], rp = Ri[K + kk];
  Ri[kk] = s * Vi[ka] + aN * rp;
  Ri[K + kk] = (-s) * Vi[K + ka] - aN * rt;
}

// Tested excitation, host medium 0 only (Eqs. 20-21 with Eq. 30), over the
// basis's two triangles in medium 0 (edge_tris, -1 when the basis does not
// bound medium 0), each triangle's piece with its side sign s0(T) (the same
// for both at an ordinary edge; they differ at a junction edge).
__global__ void k_rhs(int ne, int nrhs, const double *inc, const int *edge_tris, const int *treg,
                      const double *tri, const int *te, const double *tsg, zd k0, zd eta0, zd *b, zd aTJ, zd aNJ,
                      zd aTM, zd aNM) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (p >= ne || r >= nrhs) return;
  zd *out = b + ((size_t)r * ne + p) * 2;
  if (edge_tris[2 * p] < 0) {
    out[0] = zd();
    out[1] = zd();
    return;
  }
  double th = inc[4 * r], ph = inc[4 * r + 1], pol = inc[4 * r + 2], E0 = inc[4 * r + 3];
  double st, ct, sp, cp;
  sincos(th, &st, &ct);
  sincos(ph, &sp, &cp);
  V3 kh = v3(-st * cp, -st * sp, -ct);
  V3 e = (E0 * cos(pol)) * v3(ct * cp, ct * sp, -st) + (E0 * sin(pol)) * v3(-sp, cp, 0.0);
  V3 h = cross(kh, e);  // eta0 H times eta~_0
  zd ie0 = zd(eta0.re, -eta0.im) * (1.0 / (eta0.re * eta0.re + eta0.im * eta0.im));
  zd fE, fH, fnH, fnE;
  for (int s = 0; s < 2; ++s) {
    int t = edge_tris[2 * p + s];
    const double s0 = treg[2 * t] == 0 ? 1.0 : -1.0;
    Tri T;
    load_tri(tri, te, tsg, t, T);
    int li = 0;
    for (int a = 0; a < 3; ++a)
      if (T.e[a] == p) li = a;
    for (int a = 0; a < 7; ++a) {
      V3 rr = bary(T, c_rb[a][0], c_rb[a][1], c_rb[a][2]);
      double W = T.A * c_rw[a];
      V3 f = T.c[li] * (rr - T.fr[li]);
      zd ph_ = expmjkR(k0, dot(kh, rr));  // exp(-j k0 khat.r)
      zd w = W * ph_;
      fE += (s0 * dot(f, e)) * w;
      fH += ((s0 * dot(f, h)) * w) * ie0;
      fnH += (dot(f, cross(T.n, h)) * w) * ie0;
      fnE += dot(f, cross(T.n, e)) * w;
    }
  }
  out[0] = aTJ * (fE * ie0) + aNJ * fnH;
  out[1] = aTM * (eta0 * fH) - aNM * fnE;
}

// Far field (Eqs. 27-29), in two steps.  (1) Surface currents at the
// quadrature points of every host-medium triangle, weights folded in:
//   J_q = sum over the triangle's edges of s0 c_J W_q f_e(r_q),  M_q alike with c_M
// (f_e the RWG function of Eq. 22, s0 = +-1 the side of the host medium).
// (2) Radiation integrals N = sum_q exp(j k0 rhat.r_q) J_q, L alike with M_q,
// per observation direction; the sum over points is split into NS parts
// added in a fixed order by k_farfield_sum, which forms sigma.
__global__ void k_quad_currents(int ntri0, int ne, int nrhs, const int *__restrict__ tri0, const zd *__restrict__ x,
                                const int *__restrict__ treg, const double *__restrict__ tri,
                                const int *__restrict__ te, const double *__restrict__ tsg, double *qpos, zd *qcur) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (triangle, point)
  const int r = blockIdx.y;
  const int npts = ntri0 * 7;
  if (i >= npts) return;
  const int t = tri0[i / 7], a = i % 7;
  Tri T;
  load_tri(tri, te, tsg, t, T);
  const V3 rr = bary(T, c_rb[a][0], c_rb[a][1], c_rb[a][2]);
  const double W = T.A * c_rw[a];
  if (r == 0) {
    qpos[4 * (size_t)i] = rr.x;
    qpos[4 * (size_t)i + 1] = rr.y;
    qpos[4 * (size_t)i + 2] = rr.z;
    qpos[4 * (size_t)i + 3] = 0.0;
  }
  zd J[3], M[3];
  const double w = (treg[2 * t] == 0 ? 1.0 : -1.0) * W;  // the side of medium 0 (per triangle: also at junctions)
  for (int k = 0; k < 3; ++k) {
    const int e = T.e[k];
    if (e < 0) continue;
    const zd cJ = x[((size_t)r * ne + e) * 2], cM = x[((size_t)r * ne + e) * 2 + 1];
    const V3 f = T.c[k] * (rr - T.fr[k]);
    const double fw[3] = {w * f.x, w * f.y, w * f.z};
    for (int d = 0; d < 3; ++d) {
      J[d] += fw[d] * cJ;
      M[d] += fw[d] * cM;
    }
  }
  zd *o = qcur + ((size_t)r * npts + i) * 6;
  for (int d = 0; d < 3; ++d) {
    o[d] = J[d];
    o[3 + d] = M[d];
  }
}

constexpr int FF_TP = 64;  // points per shared-memory tile
__global__ void __launch_bounds__(128) k_farfield_part(int npts, int nobs, const double *__restrict__ obs,
                                                       const double *__restrict__ qpos, const zd *__restrict__ qcur,
                                                       zd k0, zd *part) {
  __shared__ double sp[FF_TP][4];
  __shared__ double2 sc_raw[FF_TP * 6];  // raw storage: zd has a constructor
  zd(*sc)[6] = reinterpret_cast<zd(*)[6]>(sc_raw);
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y, NS = gridDim.y, r = blockIdx.z;
  V3 rh = v3(0.0, 0.0, 0.0);
  if (o < nobs) {
    double st, ct, sp_, cp;
    sincos(obs[2 * o], &st, &ct);
    sincos(obs[2 * o + 1], &sp_, &cp);
    rh = v3(st * cp, st * sp_, ct);
  }
  const int p0 = (int)((int64_t)s * npts / NS), p1 = (int)((int64_t)(s + 1) * npts / NS);
  const zd *qc = qcur + (size_t)r * npts * 6;
  zd acc[6];
  for (int base = p0; base < p1; base += FF_TP) {
    const int cnt = min(FF_TP, p1 - base);
    __syncthreads();
    for (int idx = threadIdx.x; idx < cnt * 4; idx += blockDim.x) sp[idx / 4][idx % 4] = qpos[4 * (size_t)base + idx];
    for (int idx = threadIdx.x; idx < cnt * 6; idx += blockDim.x) sc[idx / 6][idx % 6] = qc[6 * (size_t)base + idx];
    __syncthreads();
    if (o < nobs) {
      for (int q = 0; q < cnt; ++q) {
        const double xx = rh.x * sp[q][0] + rh.y * sp[q][1] + rh.z * sp[q][2];
        double s1, c1;
        sincos(k0.re * xx, &s1, &c1);
        zd e(c1, s1);  // exp(+j k0 rhat.r)
        if (k0.im != 0.0) e = exp(-k0.im * xx) * e;
#pragma unroll
        for (int m = 0; m < 6; ++m) acc[m] += e * sc[q][m];
      }
    }
  }
  if (o < nobs) {
    zd *d = part + (((size_t)r * NS + s) * nobs + o) * 6;
    for (int m = 0; m < 6; ++m) d[m] = acc[m];
  }
}

// Mixed form (FP32 far field, the chosen precision of the excitation/RCS
// step): positions relative to the tree centre r0 and currents in FP32, the
// phase exp(j k0 rhat.(r - r0)) in FP32 with FP32 accumulation inside a
// split; the splits are added in FP64 and k_farfield_sum restores the common
// factor exp(j k0 rhat.r0).
__global__ void __launch_bounds__(128) k_farfield_part32(int npts, int nobs, const double *__restrict__ obs,
                                                         const double *__restrict__ qpos, const zd *__restrict__ qcur,
                                                         double r0x, double r0y, double r0z, zd k0, zd *part) {
  __shared__ float4 sp[FF_TP];
  __shared__ float2 sc_raw[FF_TP * 6];  // raw storage: zf has a constructor
  zf(*sc)[6] = reinterpret_cast<zf(*)[6]>(sc_raw);
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y, NS = gridDim.y, r = blockIdx.z;
  float rx = 0.f, ry = 0.f, rz = 0.f;
  if (o < nobs) {
    double st, ct, sp_, cp;
    sincos(obs[2 * o], &st, &ct);
    sincos(obs[2 * o + 1], &sp_, &cp);
    rx = (float)(st * cp);
    ry = (float)(st * sp_);
    rz = (float)ct;
  }
  const float kr = (float)k0.re, ki = (float)k0.im;
  const int p0 = (int)((int64_t)s * npts / NS), p1 = (int)((int64_t)(s + 1) * npts / NS);
  const zd *qc = qcur + (size_t)r * npts * 6;
  zf acc[6];
  for (int base = p0; base < p1; base += FF_TP) {
    const int cnt = min(FF_TP, p1 - base);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const double *pp = qpos + 4 * (size_t)(base + q);
      sp[q] = make_float4((float)(pp[0] - r0x), (float)(pp[1] - r0y), (float)(pp[2] - r0z), 0.f);
    }
    for (int idx = threadIdx.x; idx < cnt * 6; idx += blockDim.x) {
      const zd v = qc[6 * (size_t)base + idx];
      sc[idx / 6][idx % 6] = zf((float)v.re, (float)v.im);
    }
    __syncthreads();
    if (o < nobs) {
      for (int q = 0; q < cnt; ++q) {
        const float4 pq = sp[q];
        const float xx = rx * pq.x + ry * pq.y + rz * pq.z;
        float s1, c1;
        sincosf(kr * xx, &s1, &c1);
        zf e(c1, s1);
        if (ki != 0.f) e = expf(-ki * xx) * e;
#pragma unroll
        for (int m = 0; m < 6; ++m) acc[m] += e * sc[q][m];
      }
    }
  }
  if (o < nobs) {
    zd *d = part + (((size_t)r * NS + s) * nobs + o) * 6;
    for (int m = 0; m < 6; ++m) d[m] = zd(acc[m].re, acc[m].im);
  }
}

__global__ void k_farfield_sum(int nobs, int NS, const double *__restrict__ obs, const zd *__restrict__ part, zd k0,
                               zd eta0, double r0x, double r0y, double r0z, double *out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (o >= nobs) return;
  zd v[6];
  for (int s = 0; s < NS; ++s) {
    const zd *d = part + (((size_t)r * NS + s) * nobs + o) * 6;
    for (int m = 0; m < 6; ++m) v[m] += d[m];
  }
  double st, ct, sp, cp;
  sincos(obs[2 * o], &st, &ct);
  sincos(obs[2 * o + 1], &sp, &cp);
  if (r0x != 0.0 || r0y != 0.0 || r0z != 0.0) {
    // partial sums taken relative to r0: restore exp(j k0 rhat.r0)
    const double xx = st * cp * r0x + st * sp * r0y + ct * r0z;
    double s1, c1;
    sincos(k0.re * xx, &s1, &c1);
    const zd e = exp(-k0.im * xx) * zd(c1, s1);
    for (int m = 0; m < 6; ++m) v[m] = e * v[m];
  }
  const double th[3] = {ct * cp, ct * sp, -st}, ph[3] = {-sp, cp, 0.0};
  zd Nt, Np, Lt, Lp;
  for (int d = 0; d < 3; ++d) {
    Nt += th[d] * v[d];
    Np += ph[d] * v[d];
    Lt += th[d] * v[3 + d];
    Lp += ph[d] * v[3 + d];
  }
  const zd pre = zd(0.0, -1.0) * k0 * (1.0 / sqrt(4.0 * M_PI));
  const zd At = pre * (eta0 * Nt + Lp);
  const zd Ap = pre * (eta0 * Np - Lt);
  out[((size_t)r * nobs + o) * 2] = At.re * At.re + At.im * At.im;
  out[((size_t)r * nobs + o) * 2 + 1] = Ap.re * Ap.re + Ap.im * Ap.im;
}

__global__ void k_to_f32(const double *a, float *b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) b[i] = (float)a[i];
}

inline zd to_zd(std::complex<double> z) { return zd(z.real(), z.imag()); }

}  // namespace

// ------------------------------------------------------------------ launchers
void launch_near_fill(sie_ctx *c, int l) {
  upload_radon();
  RegionHost &R = c->reg[l];
  if (R.npairs == 0) return;
  int bs = 128;
  int64_t nb = (R.npairs + bs - 1) / bs;
  std::complex<double> w[4];
  form_weights(c, l, w);
  k_near_fill<<<(unsigned)nb, bs, 0, c->stream>>>(R.d_pairs, R.npairs, c->d_tri, c->d_tri_e, c->d_tri_sg,
                                                   c->d_tri_reg, l, to_zd(R.k), to_zd(R.eta), c->d_quad,
                                                   c->nq_sing, c->d_row_ptr, c->d_col, (double *)c->d_near64,
                                                   to_zd(w[0]), to_zd(w[1]), to_zd(w[2]), to_zd(w[3]));
  SIE_CHECK_LAUNCH();
  c->launches++;
}

void launch_identity(sie_ctx *c) {
  upload_radon();
  std::vector<zd> et(c->nr);
  for (int l = 0; l < c->nr; ++l) et[l] = to_zd(c->etareg[l]);
  zd *d_et = dev_upload(c, et);
  std::vector<zd> wv(4 * (size_t)c->nr);
  for (int l = 0; l < c->nr; ++l) {
    std::complex<double> w[4];
    form_weights(c, l, w);
    for (int q = 0; q < 4; ++q) wv[4 * l + q] = to_zd(w[q]);
  }
  zd *d_w = dev_upload(c, wv);
  int *d_err = (int *)dev_alloc(c, sizeof(int));
  SIE_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), c->stream));
  k_identity<<<(c->nt + 127) / 128, 128, 0, c->stream>>>(c->nt, c->d_tri, c->d_tri_e, c->d_tri_sg, c->d_tri_reg,
                                                        d_et, d_w, c->d_row_ptr, c->d_col, (double *)c->d_near64,
                                                        d_err);
  SIE_CHECK_LAUNCH();
  c->launches++;
  int err = 0;
  SIE_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SIE_CUDA(cudaStreamSynchronize(c->stream));
  SIE_REQUIRE(err == 0, SIE_EINVAL, "sie_fill_nearfield: leaf boxes smaller than triangles (use fewer levels)");
}

void launch_patterns(sie_ctx *c, int l) {
  upload_radon();
  RegionHost &R = c->reg[l];
  int leaf = c->levels - 1;
  LevelHost &LL = R.lev[leaf];
  int K = LL.K;
  size_t n = (size_t)R.nb * 2 * K;
  R.d_V64 = dev_alloc(c, n * sizeof(zd));
  R.d_P64 = dev_alloc(c, n * sizeof(zd));
  R.d_V32 = dev_alloc(c, n * sizeof(zf));
  R.d_P32 = dev_alloc(c, n * sizeof(zf));
  SIE_REQUIRE(R.nb < 65536 * 8, SIE_EINVAL, "patterns: too many bases in one medium");
  for (int i0 = 0; i0 < R.nb; i0 += 65535) {
    int cnt = std::min(65535, R.nb - i0);
    dim3 grid((K + 127) / 128, cnt);
    k_patterns<<<grid, 128, 0, c->stream>>>(cnt, K, R.d_basis_p + i0, R.d_basis_box + i0, R.d_box_centre,
                                            R.d_ptri + 2 * (size_t)i0, R.d_psg + 2 * (size_t)i0, c->d_tri,
                                            c->d_tri_e, c->d_tri_sg, LL.d_dirs,
                                            to_zd(R.k), (zd *)R.d_V64 + (size_t)i0 * 2 * K,
                                            (zd *)R.d_P64 + (size_t)i0 * 2 * K);
    SIE_CHECK_LAUNCH();
    c->launches++;
  }
  for (int i0 = 0; i0 < R.nb; i0 += 65535) {
    int cnt = std::min(65535, R.nb - i0);
    dim3 grid((K + 127) / 128, cnt);
    // tangential and normal weights of the folded pattern (PMCHWT: tangential only,
    // its impedance factors are applied per row at the receive)
    const double aT = c->form == 2 ? 0.0 : 1.0, aN = (c->form == 0 || c->form == 2) ? 1.0 : 0.0;
    k_receive_fold<<<grid, 128, 0, c->stream>>>(cnt, K, LL.L, R.d_basis_sign + i0, (const zd *)R.d_V64 + (size_t)i0 * 2 * K,
                                                (zd *)R.d_P64 + (size_t)i0 * 2 * K, aT, aN);
    SIE_CHECK_LAUNCH();
    c->launches++;
  }
  launch_to_f32(c, (const double *)R.d_V64, (float *)R.d_V32, (int64_t)n * 2);
  launch_to_f32(c, (const double *)R.d_P64, (float *)R.d_P32, (int64_t)n * 2);
  build_agg_operand(c, R, K);
  build_rec_operand(c, R, K);
}

void launch_rhs(sie_ctx *c, const double *inc_dev, int nrhs, zd *b) {
  upload_radon();
  dim3 grid((c->ne + 127) / 128, nrhs);
  std::complex<double> w[4];
  form_weights(c, 0, w);
  k_rhs<<<grid, 128, 0, c->stream>>>(c->ne, nrhs, inc_dev, c->d_edge_tris, c->d_tri_reg, c->d_tri, c->d_tri_e,
                                     c->d_tri_sg, to_zd(c->kreg[0]), to_zd(c->etareg[0]), b, to_zd(w[0]),
                                     to_zd(w[1]), to_zd(w[2]), to_zd(w[3]));
  SIE_CHECK_LAUNCH();
  c->launches++;
  op_rowscale(c, b, nrhs);  // ICTF: the excitation's rows scaled like the operator's
}

void launch_farfield(sie_ctx *c, const zd *x, int nrhs, const double *obs, int nobs, double *out, sie_prec prec) {
  upload_radon();
  const int npts = c->ntri0 * 7;
  const int ob = (nobs + 127) / 128;
  // split the point sum so that the grid fills the GPU, partials kept small
  int NS = std::min(256, (152 * 4 + ob * nrhs - 1) / (ob * nrhs));
  NS = std::max(1, std::min(NS, npts / 256));
  const size_t qpos_b = ((size_t)npts * 4 * sizeof(double) + 255) / 256 * 256;
  const size_t qcur_b = ((size_t)nrhs * npts * 6 * sizeof(zd) + 255) / 256 * 256;
  const size_t part_b = (size_t)nrhs * NS * nobs * 6 * sizeof(zd);
  const size_t need = qpos_b + qcur_b + part_b;
  if (need > c->ff_bytes) {
    c->d_ff = dev_alloc(c, need);
    c->ff_bytes = need;
  }
  double *qpos = (double *)c->d_ff;
  zd *qcur = (zd *)((char *)c->d_ff + qpos_b);
  zd *part = (zd *)((char *)c->d_ff + qpos_b + qcur_b);
  const zd k0 = to_zd(c->kreg[0]), eta0 = to_zd(c->etareg[0]);
  if (npts > 0) {
    k_quad_currents<<<dim3((npts + 127) / 128, nrhs), 128, 0, c->stream>>>(
        c->ntri0, c->ne, nrhs, c->d_tri0, x, c->d_tri_reg, c->d_tri, c->d_tri_e, c->d_tri_sg, qpos, qcur);
    SIE_CHECK_LAUNCH();
    c->launches++;
  }
  double r0[3] = {0.0, 0.0, 0.0};
  if (prec == SIE_PREC_FP64) {
    k_farfield_part<<<dim3(ob, NS, nrhs), 128, 0, c->stream>>>(npts, nobs, obs, qpos, qcur, k0, part);
  } else {
    const double root = c->hleaf * (double)(1 << std::max(0, c->levels - 1));
    for (int d = 0; d < 3; ++d) r0[d] = c->origin[d] + 0.5 * root;
    k_farfield_part32<<<dim3(ob, NS, nrhs), 128, 0, c->stream>>>(npts, nobs, obs, qpos, qcur, r0[0], r0[1], r0[2],
                                                                 k0, part);
  }
  SIE_CHECK_LAUNCH();
  k_farfield_sum<<<dim3(ob, nrhs), 128, 0, c->stream>>>(nobs, NS, obs, part, k0, eta0, r0[0], r0[1], r0[2], out);
  SIE_CHECK_LAUNCH();
  c->launches += 2;
}

void launch_to_f32(sie_ctx *c, const double *src, float *dst, int64_t n) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_to_f32<<<std::max(blocks, 1), 256, 0, c->stream>>>(src, dst, n);
  SIE_CHECK_LAUNCH();
  c->launches++;
}
