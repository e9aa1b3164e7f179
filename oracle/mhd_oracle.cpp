// Plain FP64 CPU oracle of the H-M-H Strang step for 2.5D ideal MHD on periodic
// uniform Cartesian meshes (structure-preserving splitting of the paper:
// entropy-stable DGSEM hydro stage, compatible-FE magnetic stage).
//
// TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg may load this file.  It shares no code with the
// CUDA library: every rule, table and operator is written here again, in the
// most literal form (plain loops, Lagrange products, element-by-element
// assembly), so that a reader can check it against the paper by eye.
//
// Numbering of citations: section numbers of the paper and the LaTeX equation
// labels, e.g. "eq. (euler-volume-residual)".  Readings of passages that the
// paper leaves open are tagged R1..R23 and listed in the design notes.
//
// Parity unpinned (no CPU pin a plausible mistake would fail): the CFL time
// step (reading R2) and the rejection/retry scope (R3).  Both are readings the
// paper leaves open; the GPU must match the oracle on them, and the field-loop
// numbers of §4.3 tie R2 to the paper through a GPU test only.
//
// Host layouts (shared with the C-ABI of the library, because they are the
// interface, not the arithmetic):
//   DG nodal fields   [K][(p+1)^2], K = ey*nx + ex, node j*(p+1)+i (x fastest)
//   B_x (RT, x-comp)  [ny*(m+1)][nx*(m+1)]: column ex*(m+1)+a, a = GLL(m+1)
//                     node 0..m in x; row ey*(m+1)+b, b = Gauss(m) node in y
//   B_y (RT, y-comp)  same shape: column = Gauss(m) node in x, row = GLL(m+1)
//   B_z (V_h^m)       [K][(m+1)^2] at GLL(m) nodes (one value at m = 0)
//   E/J, x-comp (N)   same layout as B_y; y-comp same as B_x; z-comp (W_h^{m+1})
//                     [ny*(m+1)][nx*(m+1)] GLL(m+1) nodes 0..m per element.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORACLE_TANGENT
// Forward-mode tangent build (liboracle_tangent.so): the same source with the
// scalar type replaced by a dual number; the values it computes are those of
// the plain build bit for bit, the tangents are directional derivatives.
#include "dual.h"
typedef Dual real;
#else
typedef double real;
inline double val(double x) { return x; }
inline double tan_of(double) { return 0.0; }
inline void freeze(double&) {}
#endif
using std::exp;
using std::fabs;
using std::isfinite;
using std::log;
using std::pow;
using std::sqrt;

namespace {

typedef std::vector<real> vec;

// ---------------------------------------------------------------------------
// O1. One-dimensional rules and Lagrange bases (§3.1.3)
// ---------------------------------------------------------------------------

// Legendre P_n(x) and P_n'(x): Bonnet recurrence, P_k' = P_{k-2}' + (2k-1) P_{k-1}.
void legendre(int n, real x, real* P, real* dP) {
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  real p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  for (int k = 2; k <= n; ++k) {
    real p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    real d2 = d0 + (2.0 * k - 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

// Gauss-Legendre rule with npts points: roots of P_npts, weights 2/((1-x^2)P'^2).
void gauss_rule(int npts, vec& x, vec& w) {
  x.assign(npts, 0.0); w.assign(npts, 0.0);
  for (int i = 0; i < (npts + 1) / 2; ++i) {
    real z = std::cos(M_PI * (i + 0.75) / (npts + 0.5));
    for (int it = 0; it < 100; ++it) {
      real P, dP; legendre(npts, z, &P, &dP);
      real dz = P / dP;
      z -= dz;
      if (fabs(dz) <= 1e-16) break;
    }
    real P, dP; legendre(npts, z, &P, &dP);
    real wt = 2.0 / ((1.0 - z * z) * dP * dP);
    x[npts - 1 - i] = z; x[i] = -z;
    w[npts - 1 - i] = wt; w[i] = wt;
  }
  if (npts % 2 == 1) x[npts / 2] = 0.0;
}

// GLL rule of degree r (r+1 points): endpoints and the roots of P_r',
// weights 2/(r(r+1)P_r^2).  r = 0 is the one-point rule xi = 0, omega = 2.
void gll_rule(int r, vec& x, vec& w) {
  if (r == 0) { x.assign(1, 0.0); w.assign(1, 2.0); return; }
  x.assign(r + 1, 0.0); w.assign(r + 1, 0.0);
  x[0] = -1.0; x[r] = 1.0;
  for (int i = 1; i <= r / 2; ++i) {
    real z = std::cos(M_PI * i / r);
    for (int it = 0; it < 100; ++it) {
      real P, dP; legendre(r, z, &P, &dP);
      real d2P = (2.0 * z * dP - r * (r + 1.0) * P) / (1.0 - z * z);  // Legendre ODE
      real dz = dP / d2P;
      z -= dz;
      if (fabs(dz) <= 1e-16) break;
    }
    x[r - i] = z; x[i] = -z;
  }
  if (r % 2 == 0) x[r / 2] = 0.0;
  for (int i = 0; i <= r; ++i) {
    real P, dP; legendre(r, x[i], &P, &dP);
    w[i] = 2.0 / (r * (r + 1.0) * P * P);
  }
}

// Lagrange basis l_j on `nodes` evaluated at x (product formula).
real lag(const vec& nodes, int j, real x) {
  real v = 1.0;
  for (int k = 0; k < (int)nodes.size(); ++k)
    if (k != j) v *= (x - nodes[k]) / (nodes[j] - nodes[k]);
  return v;
}

// Derivative of l_j at x (product rule written out).
real dlag(const vec& nodes, int j, real x) {
  real s = 0.0;
  for (int l = 0; l < (int)nodes.size(); ++l) {
    if (l == j) continue;
    real t = 1.0 / (nodes[j] - nodes[l]);
    for (int k = 0; k < (int)nodes.size(); ++k)
      if (k != j && k != l) t *= (x - nodes[k]) / (nodes[j] - nodes[k]);
    s += t;
  }
  return s;
}

// ---------------------------------------------------------------------------
// Euler pieces of the hydro stage (§3.2)
// ---------------------------------------------------------------------------

// Pressure from the mechanical-energy variables (§3.2, p = (g-1)(E - |m|^2/(2 rho))).
real pressure(const real U[5], real g) {
  return (g - 1.0) * (U[4] - (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / (2.0 * U[0]));
}

// Physical Euler flux F_d(U), d = 0 (x) or 1 (y) (§3.2).
void phys_flux(int d, const real U[5], real g, real F[5]) {
  real rho = U[0], ux = U[1] / rho, uy = U[2] / rho;
  real p = pressure(U, g);
  real ud = d == 0 ? ux : uy;
  F[0] = U[1 + d];
  F[1] = U[1] * ud + (d == 0 ? p : 0.0);
  F[2] = U[2] * ud + (d == 1 ? p : 0.0);
  F[3] = U[3] * ud;
  F[4] = (U[4] + p) * ud;
}

// Logarithmic mean with the continuous extension a_L = a_R (reading R1:
// series for small (a_L-a_R)/(a_L+a_R), Ismail & Roe 2009, switch at u = 1e-4).
real log_mean(real aL, real aR) {
  real zeta = aL / aR;
  real f = (zeta - 1.0) / (zeta + 1.0);
  real u = f * f;
  real F;
  if (u < 1e-4)
    F = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0;
  else
    F = log(zeta) / (2.0 * f);
  return (aL + aR) / (2.0 * F);
}

// Chandrashekar's entropy-conservative two-point flux, 2.5D form
// (eq. euler-chandrashekar-flux), beta = rho/(2p).
void ec_flux(int d, const real UL[5], const real UR[5], real g, real F[5]) {
  real rL = UL[0], rR = UR[0];
  real uL[3] = {UL[1] / rL, UL[2] / rL, UL[3] / rL};
  real uR[3] = {UR[1] / rR, UR[2] / rR, UR[3] / rR};
  real pL = pressure(UL, g), pR = pressure(UR, g);
  real bL = rL / (2.0 * pL), bR = rR / (2.0 * pR);
  real r_avg = 0.5 * (rL + rR);
  real b_avg = 0.5 * (bL + bR);
  real u_avg[3];
  for (int c = 0; c < 3; ++c) u_avg[c] = 0.5 * (uL[c] + uR[c]);
  real u2L = uL[0] * uL[0] + uL[1] * uL[1] + uL[2] * uL[2];
  real u2R = uR[0] * uR[0] + uR[1] * uR[1] + uR[2] * uR[2];
  real u2_avg = 0.5 * (u2L + u2R);                                        // {{|u|^2}}
  real avg_u_sq = u_avg[0] * u_avg[0] + u_avg[1] * u_avg[1] + u_avg[2] * u_avg[2];  // |{{u}}|^2
  real r_log = log_mean(rL, rR);
  real b_log = log_mean(bL, bR);
  real p_hat = r_avg / (2.0 * b_avg);
  real h_hat = 1.0 / (2.0 * (g - 1.0) * b_log) - 0.5 * u2_avg + avg_u_sq + p_hat / r_log;
  real ud = u_avg[d];
  F[0] = r_log * ud;
  F[1] = r_log * u_avg[0] * ud + (d == 0 ? p_hat : 0.0);
  F[2] = r_log * u_avg[1] * ud + (d == 1 ? p_hat : 0.0);
  F[3] = r_log * u_avg[2] * ud;
  F[4] = r_log * ud * h_hat;
}

// Local Lax-Friedrichs flux (eq. euler-lf-flux) with acoustic c = sqrt(g p / rho).
void llf_flux(int d, const real Um[5], const real Up[5], real g, real F[5]) {
  real Fm[5], Fp[5];
  phys_flux(d, Um, g, Fm);
  phys_flux(d, Up, g, Fp);
  real sm = fabs(Um[1 + d] / Um[0]) + sqrt(g * pressure(Um, g) / Um[0]);
  real sp = fabs(Up[1 + d] / Up[0]) + sqrt(g * pressure(Up, g) / Up[0]);
  real lam = std::max(sm, sp);
  for (int c = 0; c < 5; ++c) F[c] = 0.5 * (Fm[c] + Fp[c]) - 0.5 * lam * (Up[c] - Um[c]);
}

struct Params {
  int oe_hydro, oe_vel, pp, ar;
  real s_H, s_M, C_s, C_eta, cfl;
  int max_halvings;
  int ec_faces;  // test hook: entropy-conservative flux on faces instead of LLF
  int frozen;    // tangent build: hold the stabilisation coefficients (D_l, theta, eta) at their values
  int strang_order;  // 0: H-M-H (eq. strang-composition, Algorithm 3); 1: M-H-M (reading R20)
};

enum { OR_OK = 0, OR_RETRIED = 1, OR_REJECT = -10, OR_INADMISSIBLE = -11 };

// ---------------------------------------------------------------------------
// The discretisation
// ---------------------------------------------------------------------------
struct Oracle {
  int nx, ny, K, p, m, n, n2, mm, mL, NX, NY;
  real x0, x1, y0, y1, hx, hy, Jdet, g;
  Params prm;
  vec xp, wp;  // GLL(p): DG nodes
  vec xL, wL;  // GLL(m+1): W nodes, continuous direction of N and R
  vec xM, wM;  // GLL(m): V_h^m nodes of B_z
  vec zG, wG;  // Gauss(m), m+1 points: discontinuous direction of N and R
  vec z2, w2;  // Gauss with m+2 points: exact RT block of the magnetic product
  vec D;       // D_ij = l_j'(xi_i) on GLL(p)
  vec U[5];    // rho, m_x, m_y, m_z, E_mech
  vec Bx, By, Bz;
  vec eta;     // element resistivity used in the last magnetic substep
  int last_rejections;

  int emod(int e, int N) const { return ((e % N) + N) % N; }
  int kid(int ex, int ey) const { return emod(ey, ny) * nx + emod(ex, nx); }
  int gidx(int X, int Y) const { return emod(Y, NY) * NX + emod(X, NX); }
  real Q(int i, int r) const { return wp[i] * D[i * n + r]; }  // Q = M D

  void init(int nx_, int ny_, real x0_, real x1_, real y0_, real y1_, int p_, int m_, real g_) {
    nx = nx_; ny = ny_; K = nx * ny; p = p_; m = m_; n = p + 1; n2 = n * n;
    mm = m + 1; mL = m + 2; NX = nx * mm; NY = ny * mm;
    x0 = x0_; x1 = x1_; y0 = y0_; y1 = y1_;
    hx = (x1 - x0) / nx; hy = (y1 - y0) / ny; Jdet = hx * hy / 4.0; g = g_;
    gll_rule(p, xp, wp);
    gll_rule(m + 1, xL, wL);
    gll_rule(m, xM, wM);
    gauss_rule(m + 1, zG, wG);
    gauss_rule(m + 2, z2, w2);
    D.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) D[i * n + j] = dlag(xp, j, xp[i]);
    for (int c = 0; c < 5; ++c) U[c].assign((size_t)K * n2, 0.0);
    Bx.assign((size_t)NX * NY, 0.0); By = Bx; Bz.assign((size_t)K * mm * mm, 0.0);
    eta.assign(K, 0.0);
    prm = Params{0, 0, 0, 0, 0.02, 0.02, 5.0, 0.0, 0.4, 20, 0, 0, 0};
    last_rejections = 0;
  }

  // ---- element closures of the compatible fields --------------------------
  // "X-type": GLL(m+1) in x (a = 0..m+1), Gauss(m) in y (b = 0..m): B_x, E_y, J_y
  void clX(const vec& A, int ex, int ey, real* c) const {
    for (int b = 0; b < mm; ++b)
      for (int a = 0; a < mL; ++a) c[b * mL + a] = A[gidx(ex * mm + a, ey * mm + b)];
  }
  // "Y-type": Gauss(m) in x (a = 0..m), GLL(m+1) in y (b = 0..m+1): B_y, E_x, J_x
  void clY(const vec& A, int ex, int ey, real* c) const {
    for (int b = 0; b < mL; ++b)
      for (int a = 0; a < mm; ++a) c[b * mm + a] = A[gidx(ex * mm + a, ey * mm + b)];
  }
  // "W-type": GLL(m+1) in both directions: E_z, J_z, potentials
  void clW(const vec& A, int ex, int ey, real* c) const {
    for (int b = 0; b < mL; ++b)
      for (int a = 0; a < mL; ++a) c[b * mL + a] = A[gidx(ex * mm + a, ey * mm + b)];
  }

  // Tensor-product evaluation sum_{a,b} c[b][a] phi_a(x) psi_b(y); dx/dy select
  // reference derivatives.
  static real ev(const real* c, const vec& nx_, const vec& ny_, real x, real y, int dx, int dy) {
    real s = 0.0;
    int na = nx_.size(), nb = ny_.size();
    real fx[16];
    for (int a = 0; a < na; ++a) fx[a] = dx ? dlag(nx_, a, x) : lag(nx_, a, x);
    for (int b = 0; b < nb; ++b) {
      real fy = dy ? dlag(ny_, b, y) : lag(ny_, b, y);
      for (int a = 0; a < na; ++a) s += c[b * na + a] * fx[a] * fy;
    }
    return s;
  }
  real evX(const real* c, real x, real y, int dx = 0, int dy = 0) const { return ev(c, xL, zG, x, y, dx, dy); }
  real evY(const real* c, real x, real y, int dx = 0, int dy = 0) const { return ev(c, zG, xL, x, y, dx, dy); }
  real evW(const real* c, real x, real y, int dx = 0, int dy = 0) const { return ev(c, xL, xL, x, y, dx, dy); }
  real evZ(const real* c, real x, real y, int dx = 0, int dy = 0) const { return ev(c, xM, xM, x, y, dx, dy); }
  real evDG(const real* c, real x, real y) const { return ev(c, xp, xp, x, y, 0, 0); }

  // B_h of element (ex,ey) at reference point (x,y).
  void B_at(const real* bx, const real* by, const real* bz, real x, real y, real B[3]) const {
    B[0] = evX(bx, x, y); B[1] = evY(by, x, y); B[2] = evZ(bz, x, y);
  }

  // ------------------------------------------------------------------------
  // Hydro residual L_E (eq. euler-nodal-index with eq. euler-volume-residual)
  // ------------------------------------------------------------------------
  void node_state(const vec* S, int k, int i, int j, real u[5]) const {
    for (int c = 0; c < 5; ++c) u[c] = S[c][(size_t)k * n2 + j * n + i];
  }
  void face_flux(int d, const real Um[5], const real Up[5], real F[5]) const {
    if (prm.ec_faces) ec_flux(d, Um, Up, g, F);
    else llf_flux(d, Um, Up, g, F);
  }

  void hydro_rhs(const vec* S, vec* L) const {
#pragma omp parallel for collapse(2) schedule(static)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        int k = kid(ex, ey);
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            real Ui[5], Ur[5], F[5], Fs[5], R[5] = {0, 0, 0, 0, 0};
            node_state(S, k, i, j, Ui);
            for (int r = 0; r < n; ++r) {  // x-direction volume term
              node_state(S, k, r, j, Ur);
              ec_flux(0, Ui, Ur, g, F);
              for (int c = 0; c < 5; ++c) R[c] += 2.0 * Q(i, r) * wp[j] * (hy / 2.0) * F[c];
            }
            for (int s = 0; s < n; ++s) {  // y-direction volume term
              node_state(S, k, i, s, Ur);
              ec_flux(1, Ui, Ur, g, F);
              for (int c = 0; c < 5; ++c) R[c] += 2.0 * wp[i] * Q(j, s) * (hx / 2.0) * F[c];
            }
            // interface terms: Delta F~ = F~ - F~*, traces ordered in +x / +y
            if (i == 0) {
              real Um[5]; node_state(S, kid(ex - 1, ey), p, j, Um);
              face_flux(0, Um, Ui, Fs); phys_flux(0, Ui, g, F);
              for (int c = 0; c < 5; ++c) R[c] += wp[j] * (hy / 2.0) * (F[c] - Fs[c]);
            }
            if (i == p) {
              real Up[5]; node_state(S, kid(ex + 1, ey), 0, j, Up);
              face_flux(0, Ui, Up, Fs); phys_flux(0, Ui, g, F);
              for (int c = 0; c < 5; ++c) R[c] -= wp[j] * (hy / 2.0) * (F[c] - Fs[c]);
            }
            if (j == 0) {
              real Um[5]; node_state(S, kid(ex, ey - 1), i, p, Um);
              face_flux(1, Um, Ui, Fs); phys_flux(1, Ui, g, F);
              for (int c = 0; c < 5; ++c) R[c] += wp[i] * (hx / 2.0) * (F[c] - Fs[c]);
            }
            if (j == p) {
              real Up[5]; node_state(S, kid(ex, ey + 1), i, 0, Up);
              face_flux(1, Ui, Up, Fs); phys_flux(1, Ui, g, F);
              for (int c = 0; c < 5; ++c) R[c] -= wp[i] * (hx / 2.0) * (F[c] - Fs[c]);
            }
            real M = Jdet * wp[i] * wp[j];
            for (int c = 0; c < 5; ++c) L[c][(size_t)k * n2 + j * n + i] = -R[c] / M;
          }
      }
  }

  // Quadrature-weighted element average (eq. euler-pp-average): sum M U / |K|.
  void element_average(const vec* S, int k, real avg[5]) const {
    for (int c = 0; c < 5; ++c) {
      real s = 0.0;
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) s += Jdet * wp[i] * wp[j] * S[c][(size_t)k * n2 + j * n + i];
      avg[c] = s / (4.0 * Jdet);
    }
  }

  // Raw-average admissibility check before the stage map (§3.2.3, reading R9).
  bool averages_admissible(const vec* S) const {
    for (int k = 0; k < K; ++k) {
      real a[5]; element_average(S, k, a);
      bool finite = true;
      for (int c = 0; c < 5; ++c) finite = finite && isfinite(a[c]);
      if (!finite || !(a[0] > 0.0) || !(pressure(a, g) > 0.0)) return false;
    }
    return true;
  }

  // Stage map P = P_PP o P_OE (eq. euler-stage-map); the pieces are below.
  void hydro_stage_map(vec* S, real tau);

  // Hydro substep Phi_H^tau (Algorithm 1, eq. euler-ssprk33).
  int hydro_substep(real tau) {
    vec U0[5], S[5], L[5], C[5];
    for (int c = 0; c < 5; ++c) { U0[c] = U[c]; S[c] = U[c]; L[c].assign(U[c].size(), 0.0); C[c] = U[c]; }
    const real a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int s = 0; s < 3; ++s) {
      hydro_rhs(S, L);
      for (int c = 0; c < 5; ++c)
        for (size_t q = 0; q < C[c].size(); ++q) {
          real raw = S[c][q] + tau * L[c][q];
          C[c][q] = (s == 0) ? raw : a[s] * U0[c][q] + b[s] * raw;
        }
      if (!averages_admissible(C)) return OR_REJECT;
      hydro_stage_map(C, tau);
      for (int c = 0; c < 5; ++c) S[c] = C[c];
    }
    for (int c = 0; c < 5; ++c) U[c] = S[c];
    return OR_OK;
  }

  // ------------------------------------------------------------------------
  // Magnetic stage (§3.3): Y = (e, u, B) with rho frozen.
  // ------------------------------------------------------------------------
  struct Mag { vec e, u[3], Bx, By, Bz; };

  // Current J_h from the weak curl (eq. mag-current-proj): lumped A-product
  // (eq. aux-inner-product) on the left, exact magnetic product
  // (eq. magnetic-inner-product) on the right, assembled over the elements.
  // The element loads are independent (the OpenMP timing build spreads them
  // over threads); the assembly adds them in element order, so every build
  // gives the same sums bit for bit.
  void compute_J(const vec& bX, const vec& bY, const vec& bZ, vec& Jx, vec& Jy, vec& Jz) const {
    size_t G = (size_t)NX * NY;
    vec lx(G, 0.0), ly(G, 0.0), lz(G, 0.0), mx(G, 0.0), my(G, 0.0), mz(G, 0.0);
    const size_t nW = (size_t)mL * mL, nNx = (size_t)mL * mm, nNy = (size_t)mm * mL;
    vec LW((size_t)K * nW), LNx((size_t)K * nNx), LNy((size_t)K * nNy);
#pragma omp parallel
    {
      std::vector<real> bx(mL * mm), by(mm * mL);
      std::vector<real> bxq(mL * mL), byq(mL * mL), bzq(mm * mm);
      std::vector<real> Lq(mL * mL), dLq(mL * mL);
#pragma omp for collapse(2) schedule(static)
      for (int ey = 0; ey < ny; ++ey)
        for (int ex = 0; ex < nx; ++ex) {
          int k = kid(ex, ey);
          clX(bX, ex, ey, bx.data()); clY(bY, ex, ey, by.data());
          const real* bz = &bZ[(size_t)k * mm * mm];
          // W block: (J_z, phi)_W = (B_x, d_y phi)_B - (B_y, d_x phi)_B
          for (int qy = 0; qy < mL; ++qy)
            for (int qx = 0; qx < mL; ++qx) {
              bxq[qy * mL + qx] = evX(bx.data(), z2[qx], z2[qy]);
              byq[qy * mL + qx] = evY(by.data(), z2[qx], z2[qy]);
            }
          for (int qy = 0; qy < mm; ++qy)
            for (int qx = 0; qx < mm; ++qx) bzq[qy * mm + qx] = evZ(bz, zG[qx], zG[qy]);
          // GLL(m+1) basis and derivative at the Gauss(m+2) points
          for (int a = 0; a < mL; ++a)
            for (int q = 0; q < mL; ++q) { Lq[a * mL + q] = lag(xL, a, z2[q]); dLq[a * mL + q] = dlag(xL, a, z2[q]); }
          for (int b = 0; b < mL; ++b)
            for (int a = 0; a < mL; ++a) {
              real s = 0.0;
              for (int qy = 0; qy < mL; ++qy)
                for (int qx = 0; qx < mL; ++qx) {
                  real dyphi = (2.0 / hy) * Lq[a * mL + qx] * dLq[b * mL + qy];
                  real dxphi = (2.0 / hx) * dLq[a * mL + qx] * Lq[b * mL + qy];
                  s += Jdet * w2[qx] * w2[qy] * (bxq[qy * mL + qx] * dyphi - byq[qy * mL + qx] * dxphi);
                }
              LW[k * nW + b * mL + a] = s;
            }
          // N block, x-component: DOF g_a(x) l_b(y) e_x; (J_x, phi)_N = (B_z, -d_y phi)_B
          for (int b = 0; b < mL; ++b)
            for (int a = 0; a < mm; ++a) {
              real s = 0.0;
              for (int qy = 0; qy < mm; ++qy)
                for (int qx = 0; qx < mm; ++qx) {
                  real X = zG[qx], Y = zG[qy];
                  real dyphi = (2.0 / hy) * lag(zG, a, X) * dlag(xL, b, Y);
                  s += Jdet * wG[qx] * wG[qy] * bzq[qy * mm + qx] * (-dyphi);
                }
              LNx[k * nNx + b * mm + a] = s;
            }
          // N block, y-component: DOF l_a(x) g_b(y) e_y; (J_y, phi)_N = (B_z, d_x phi)_B
          for (int b = 0; b < mm; ++b)
            for (int a = 0; a < mL; ++a) {
              real s = 0.0;
              for (int qy = 0; qy < mm; ++qy)
                for (int qx = 0; qx < mm; ++qx) {
                  real X = zG[qx], Y = zG[qy];
                  real dxphi = (2.0 / hx) * dlag(xL, a, X) * lag(zG, b, Y);
                  s += Jdet * wG[qx] * wG[qy] * bzq[qy * mm + qx] * dxphi;
                }
              LNy[k * nNy + b * mL + a] = s;
            }
        }
    }
    // assembly over the elements sharing each DOF (element order)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        size_t k = (size_t)kid(ex, ey);
        for (int b = 0; b < mL; ++b)
          for (int a = 0; a < mL; ++a) {
            size_t gi = gidx(ex * mm + a, ey * mm + b);
            lz[gi] += LW[k * nW + b * mL + a]; mz[gi] += Jdet * wL[a] * wL[b];
          }
        for (int b = 0; b < mL; ++b)
          for (int a = 0; a < mm; ++a) {
            size_t gi = gidx(ex * mm + a, ey * mm + b);
            lx[gi] += LNx[k * nNx + b * mm + a]; mx[gi] += Jdet * wG[a] * wL[b];
          }
        for (int b = 0; b < mm; ++b)
          for (int a = 0; a < mL; ++a) {
            size_t gi = gidx(ex * mm + a, ey * mm + b);
            ly[gi] += LNy[k * nNy + b * mL + a]; my[gi] += Jdet * wL[a] * wG[b];
          }
      }
    Jx.assign(G, 0.0); Jy.assign(G, 0.0); Jz.assign(G, 0.0);
    for (size_t q = 0; q < G; ++q) { Jx[q] = lx[q] / mx[q]; Jy[q] = ly[q] / my[q]; Jz[q] = lz[q] / mz[q]; }
  }

  // Electric field from the lumped Ohm law (eq. mag-electric-proj):
  // (E, G)_A = C_h(u, B; G) + (eta J.G, 1)_V, C_h = (-u x B, G)_A evaluated
  // element by element at the auxiliary nodes (reading R12); the resistive load
  // uses the DG-GLL(p) rule (reading R13).
  void compute_E(const vec* u, const vec& bX, const vec& bY, const vec& bZ, const vec& etaK,
                 const vec& Jx, const vec& Jy, const vec& Jz, vec& Ex, vec& Ey, vec& Ez) const {
    size_t G = (size_t)NX * NY;
    vec lx(G, 0.0), ly(G, 0.0), lz(G, 0.0), mx(G, 0.0), my(G, 0.0), mz(G, 0.0);
    // element loads (independent; spread over threads in the OpenMP timing
    // build), then the assembly in element order as for J_h
    const size_t nNx = (size_t)mL * mm, nNy = (size_t)mm * mL, nW = (size_t)mL * mL;
    vec LNx((size_t)K * nNx), LNy((size_t)K * nNy), LW((size_t)K * nW);
#pragma omp parallel
    {
      std::vector<real> bx(mL * mm), by(mm * mL), jx(mm * mL), jy(mL * mm), jz(mL * mL);
#pragma omp for collapse(2) schedule(static)
      for (int ey = 0; ey < ny; ++ey)
        for (int ex = 0; ex < nx; ++ex) {
          int k = kid(ex, ey);
          clX(bX, ex, ey, bx.data()); clY(bY, ex, ey, by.data());
          clY(Jx, ex, ey, jx.data()); clX(Jy, ex, ey, jy.data()); clW(Jz, ex, ey, jz.data());
          const real* bz = &bZ[(size_t)k * mm * mm];
          const real* ux = &u[0][(size_t)k * n2];
          const real* uy = &u[1][(size_t)k * n2];
          const real* uz = &u[2][(size_t)k * n2];
          real ek = etaK[k];
          // resistive field J_h at the DG-GLL(p) nodes of this element
          std::vector<real> Jq(3 * n2);
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              Jq[0 * n2 + j * n + i] = evY(jx.data(), xp[i], xp[j]);
              Jq[1 * n2 + j * n + i] = evX(jy.data(), xp[i], xp[j]);
              Jq[2 * n2 + j * n + i] = evW(jz.data(), xp[i], xp[j]);
            }
          // x-component at N_x nodes (zeta_a, xi^L_b)
          for (int b = 0; b < mL; ++b)
            for (int a = 0; a < mm; ++a) {
              real X = zG[a], Y = xL[b], B[3];
              B_at(bx.data(), by.data(), bz, X, Y, B);
              real vy = evDG(uy, X, Y), vz = evDG(uz, X, Y);
              real val = -(vy * B[2] - vz * B[1]);
              real w = Jdet * wG[a] * wL[b];
              real load = w * val;
              if (ek != 0.0) {
                real r = 0.0;
                for (int j = 0; j < n; ++j)
                  for (int i = 0; i < n; ++i)
                    r += Jdet * wp[i] * wp[j] * Jq[0 * n2 + j * n + i] * lag(zG, a, xp[i]) * lag(xL, b, xp[j]);
                load += ek * r;
              }
              LNx[k * nNx + b * mm + a] = load;
            }
          // y-component at N_y nodes (xi^L_a, zeta_b)
          for (int b = 0; b < mm; ++b)
            for (int a = 0; a < mL; ++a) {
              real X = xL[a], Y = zG[b], B[3];
              B_at(bx.data(), by.data(), bz, X, Y, B);
              real vx = evDG(ux, X, Y), vz = evDG(uz, X, Y);
              real val = -(vz * B[0] - vx * B[2]);
              real w = Jdet * wL[a] * wG[b];
              real load = w * val;
              if (ek != 0.0) {
                real r = 0.0;
                for (int j = 0; j < n; ++j)
                  for (int i = 0; i < n; ++i)
                    r += Jdet * wp[i] * wp[j] * Jq[1 * n2 + j * n + i] * lag(xL, a, xp[i]) * lag(zG, b, xp[j]);
                load += ek * r;
              }
              LNy[k * nNy + b * mL + a] = load;
            }
          // z-component at W nodes (xi^L_a, xi^L_b)
          for (int b = 0; b < mL; ++b)
            for (int a = 0; a < mL; ++a) {
              real X = xL[a], Y = xL[b], B[3];
              B_at(bx.data(), by.data(), bz, X, Y, B);
              real vx = evDG(ux, X, Y), vy = evDG(uy, X, Y);
              real val = -(vx * B[1] - vy * B[0]);
              real w = Jdet * wL[a] * wL[b];
              real load = w * val;
              if (ek != 0.0) {
                real r = 0.0;
                for (int j = 0; j < n; ++j)
                  for (int i = 0; i < n; ++i)
                    r += Jdet * wp[i] * wp[j] * Jq[2 * n2 + j * n + i] * lag(xL, a, xp[i]) * lag(xL, b, xp[j]);
                load += ek * r;
              }
              LW[k * nW + b * mL + a] = load;
            }
        }
    }
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        size_t k = (size_t)kid(ex, ey);
        for (int b = 0; b < mL; ++b)
          for (int a = 0; a < mm; ++a) {
            size_t gi = gidx(ex * mm + a, ey * mm + b);
            lx[gi] += LNx[k * nNx + b * mm + a]; mx[gi] += Jdet * wG[a] * wL[b];
          }
        for (int b = 0; b < mm; ++b)
          for (int a = 0; a < mL; ++a) {
            size_t gi = gidx(ex * mm + a, ey * mm + b);
            ly[gi] += LNy[k * nNy + b * mL + a]; my[gi] += Jdet * wL[a] * wG[b];
          }
        for (int b = 0; b < mL; ++b)
          for (int a = 0; a < mL; ++a) {
            size_t gi = gidx(ex * mm + a, ey * mm + b);
            lz[gi] += LW[k * nW + b * mL + a]; mz[gi] += Jdet * wL[a] * wL[b];
          }
      }
    Ex.assign(G, 0.0); Ey.assign(G, 0.0); Ez.assign(G, 0.0);
    for (size_t q = 0; q < G; ++q) { Ex[q] = lx[q] / mx[q]; Ey[q] = ly[q] / my[q]; Ez[q] = lz[q] / mz[q]; }
  }

  // Magnetic residual L_M (eq. magnetic-dae): returns de, du, dB.
  void mag_rhs(const vec& rho, const vec& etaK, const Mag& Y, Mag& dY, vec* Jout = nullptr, vec* Eout = nullptr) const {
    vec Jx, Jy, Jz, Ex, Ey, Ez;
    compute_J(Y.Bx, Y.By, Y.Bz, Jx, Jy, Jz);
    compute_E(Y.u, Y.Bx, Y.By, Y.Bz, etaK, Jx, Jy, Jz, Ex, Ey, Ez);
    if (Jout) { Jout[0] = Jx; Jout[1] = Jy; Jout[2] = Jz; }
    if (Eout) { Eout[0] = Ex; Eout[1] = Ey; Eout[2] = Ez; }
    size_t G = (size_t)NX * NY;
    dY.e.assign((size_t)K * n2, 0.0);
    for (int d = 0; d < 3; ++d) dY.u[d].assign((size_t)K * n2, 0.0);
    dY.Bx.assign(G, 0.0); dY.By.assign(G, 0.0); dY.Bz.assign((size_t)K * mm * mm, 0.0);
    // every element writes only its own DOFs and nodes (threads in the OpenMP timing build)
#pragma omp parallel
    {
    std::vector<real> bx(mL * mm), by(mm * mL), jx(mm * mL), jy(mL * mm), jz(mL * mL),
        exc(mm * mL), eyc(mL * mm), ezc(mL * mL);
#pragma omp for collapse(2) schedule(static)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        int k = kid(ex, ey);
        clX(Y.Bx, ex, ey, bx.data()); clY(Y.By, ex, ey, by.data());
        clY(Jx, ex, ey, jx.data()); clX(Jy, ex, ey, jy.data()); clW(Jz, ex, ey, jz.data());
        clY(Ex, ex, ey, exc.data()); clX(Ey, ex, ey, eyc.data()); clW(Ez, ex, ey, ezc.data());
        const real* bz = &Y.Bz[(size_t)k * mm * mm];
        // -curl E on the DOFs owned by this element: dB_par = grad^perp E_z
        for (int b = 0; b < mm; ++b)
          for (int a = 0; a < mm; ++a) {
            dY.Bx[gidx(ex * mm + a, ey * mm + b)] = -(2.0 / hy) * evW(ezc.data(), xL[a], zG[b], 0, 1);
            dY.By[gidx(ex * mm + a, ey * mm + b)] = (2.0 / hx) * evW(ezc.data(), zG[a], xL[b], 1, 0);
            real dEy_dx = (2.0 / hx) * evX(eyc.data(), xM[a], xM[b], 1, 0);
            real dEx_dy = (2.0 / hy) * evY(exc.data(), xM[a], xM[b], 0, 1);
            dY.Bz[(size_t)k * mm * mm + b * mm + a] = -(dEy_dx - dEx_dy);
          }
        // Lorentz load: algebraic transpose of C_h (eq. semi-vel), Ohmic heating (eq. ohmic-heating)
        // B_h of this element at its auxiliary nodes (N_x, N_y and W families)
        std::vector<real> Bnx(3 * mL * mm), Bny(3 * mL * mm), Bw(3 * mL * mL);
        for (int b = 0; b < mL; ++b)
          for (int a = 0; a < mm; ++a) B_at(bx.data(), by.data(), bz, zG[a], xL[b], &Bnx[3 * (b * mm + a)]);
        for (int b = 0; b < mm; ++b)
          for (int a = 0; a < mL; ++a) B_at(bx.data(), by.data(), bz, xL[a], zG[b], &Bny[3 * (b * mL + a)]);
        for (int b = 0; b < mL; ++b)
          for (int a = 0; a < mL; ++a) B_at(bx.data(), by.data(), bz, xL[a], xL[b], &Bw[3 * (b * mL + a)]);
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            real sx = 0.0, sy = 0.0, sz = 0.0;
            for (int b = 0; b < mL; ++b)  // N_x nodes
              for (int a = 0; a < mm; ++a) {
                real X = zG[a], Yq = xL[b];
                const real* B = &Bnx[3 * (b * mm + a)];
                real w = Jdet * wG[a] * wL[b] * lag(xp, i, X) * lag(xp, j, Yq);
                real jv = jx[b * mm + a];
                sy += -w * B[2] * jv;
                sz += w * B[1] * jv;
              }
            for (int b = 0; b < mm; ++b)  // N_y nodes
              for (int a = 0; a < mL; ++a) {
                real X = xL[a], Yq = zG[b];
                const real* B = &Bny[3 * (b * mL + a)];
                real w = Jdet * wL[a] * wG[b] * lag(xp, i, X) * lag(xp, j, Yq);
                real jv = jy[b * mL + a];
                sx += w * B[2] * jv;
                sz += -w * B[0] * jv;
              }
            for (int b = 0; b < mL; ++b)  // W nodes
              for (int a = 0; a < mL; ++a) {
                real X = xL[a], Yq = xL[b];
                const real* B = &Bw[3 * (b * mL + a)];
                real w = Jdet * wL[a] * wL[b] * lag(xp, i, X) * lag(xp, j, Yq);
                real jv = jz[b * mL + a];
                sx += -w * B[1] * jv;
                sy += w * B[0] * jv;
              }
            size_t q = (size_t)k * n2 + j * n + i;
            real M = Jdet * wp[i] * wp[j];
            dY.u[0][q] = sx / (rho[q] * M);
            dY.u[1][q] = sy / (rho[q] * M);
            dY.u[2][q] = sz / (rho[q] * M);
            real jxq = evY(jx.data(), xp[i], xp[j]);
            real jyq = evX(jy.data(), xp[i], xp[j]);
            real jzq = evW(jz.data(), xp[i], xp[j]);
            dY.e[q] = etaK[k] * (jxq * jxq + jyq * jyq + jzq * jzq) / rho[q];
          }
      }
    }
  }

  // Stabilisation pieces of the magnetic stage (velocity OE and A.R.).
  void B_at_dg_state(const Mag& Y, int ex, int ey, int i, int j, real B[3]) const;
  void ar_coefficient(const vec& rho, const Mag& Y, vec& etaK) const;
  struct VelProj;
  void vel_oe(const vec& rho, Mag& Y, real tau, const VelProj* P) const;

  // Magnetic substep Phi_M^tau (Algorithm 2, eq. magnetic-ssprk33).
  int mag_substep(const vec& rho, Mag& Y, real tau);

  // Nodal exchange (§3.4.1).
  void cons_to_prim(Mag& Y) const {
    size_t N = (size_t)K * n2;
    Y.e.assign(N, 0.0);
    for (int d = 0; d < 3; ++d) Y.u[d].assign(N, 0.0);
    for (size_t q = 0; q < N; ++q) {
      real rho = U[0][q];
      real ux = U[1][q] / rho, uy = U[2][q] / rho, uz = U[3][q] / rho;
      Y.u[0][q] = ux; Y.u[1][q] = uy; Y.u[2][q] = uz;
      Y.e[q] = (U[4][q] - 0.5 * rho * (ux * ux + uy * uy + uz * uz)) / rho;
    }
    Y.Bx = Bx; Y.By = By; Y.Bz = Bz;
  }
  void prim_to_cons(const Mag& Y) {
    size_t N = (size_t)K * n2;
    for (size_t q = 0; q < N; ++q) {
      real rho = U[0][q];
      real ux = Y.u[0][q], uy = Y.u[1][q], uz = Y.u[2][q];
      U[1][q] = rho * ux; U[2][q] = rho * uy; U[3][q] = rho * uz;
      U[4][q] = rho * Y.e[q] + 0.5 * rho * (ux * ux + uy * uy + uz * uz);
    }
    Bx = Y.Bx; By = Y.By; Bz = Y.Bz;
  }

  int run_mag(real tau) {
    Mag Y; cons_to_prim(Y);
    vec rho = U[0];
    int st = mag_substep(rho, Y, tau);
    prim_to_cons(Y);
    return st;
  }

  // One Strang step (Algorithm 3, eq. strang-composition) with the rejection
  // and retry of reading R3.
  int strang_step(real dt, real* dt_taken) {
    vec U0[5]; for (int c = 0; c < 5; ++c) U0[c] = U[c];
    vec B0x = Bx, B0y = By, B0z = Bz;
    last_rejections = 0;
    for (int att = 0; att <= prm.max_halvings; ++att) {
      int st;
      if (prm.strang_order == 1) {  // Phi_M^{dt/2} o Phi_H^{dt} o Phi_M^{dt/2} (reading R20)
        st = run_mag(0.5 * dt);
        if (st == OR_OK) st = hydro_substep(dt);
        if (st == OR_OK) st = run_mag(0.5 * dt);
      } else {  // Phi_H^{dt/2} o Phi_M^{dt} o Phi_H^{dt/2}
        st = hydro_substep(0.5 * dt);
        if (st == OR_OK) st = run_mag(dt);
        if (st == OR_OK) st = hydro_substep(0.5 * dt);
      }
      if (st == OR_OK) {
        if (dt_taken) *dt_taken = dt;
        return att > 0 ? OR_RETRIED : OR_OK;
      }
      for (int c = 0; c < 5; ++c) U[c] = U0[c];
      Bx = B0x; By = B0y; Bz = B0z;
      last_rejections++;
      dt *= 0.5;
    }
    if (dt_taken) *dt_taken = 0.0;
    return OR_INADMISSIBLE;
  }

  // B_h at the DG node (i,j) of element (ex,ey).
  void B_at_dg(int ex, int ey, int i, int j, real B[3]) const {
    std::vector<real> bx(mL * mm), by(mm * mL);
    clX(Bx, ex, ey, bx.data()); clY(By, ex, ey, by.data());
    B_at(bx.data(), by.data(), &Bz[(size_t)kid(ex, ey) * mm * mm], xp[i], xp[j], B);
  }

  // CFL time step (reading R2): the paper gives the CFL number, not the
  // formula.  Parity unpinned: no CPU pin fixes this formula; the GPU matches
  // it to rounding, and the paper's field-loop numbers (§4.3) select it only
  // through a GPU test of whole runs.
  real cfl_dt() const {
    real mx = 0.0;
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        int k = kid(ex, ey);
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            real Ui[5]; node_state(U, k, i, j, Ui);
            real B[3]; B_at_dg(ex, ey, i, j, B);
            real rho = Ui[0], pr = pressure(Ui, g);
            real cf = sqrt((g * pr + B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho);
            real r = (2.0 * p + 1.0) * std::max((fabs(Ui[1] / rho) + cf) / hx, (fabs(Ui[2] / rho) + cf) / hy);
            mx = std::max(mx, r);
          }
      }
    return prm.cfl / mx;
  }

  // B_h||_{Gauss(m)^2} divergence metric (reading R16): max over elements of
  // min(hx,hy) * max |dBx/dx + dBy/dy| at the Gauss(m) points.
  real div_metric() const {
    real mx = 0.0;
    std::vector<real> bx(mL * mm), by(mm * mL);
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        clX(Bx, ex, ey, bx.data()); clY(By, ex, ey, by.data());
        for (int b = 0; b < mm; ++b)
          for (int a = 0; a < mm; ++a) {
            real dv = (2.0 / hx) * evX(bx.data(), zG[a], zG[b], 1, 0) + (2.0 / hy) * evY(by.data(), zG[a], zG[b], 0, 1);
            mx = std::max(mx, std::min(hx, hy) * fabs(dv));
          }
      }
    return mx;
  }

  // Magnetic energy 1/2 (B,B)_B with the exact product (eq. magnetic-inner-product).
  real mag_energy(const vec& bX, const vec& bY, const vec& bZ, const vec* cX = nullptr, const vec* cY = nullptr,
                    const vec* cZ = nullptr) const {
    // returns (B, C)_B; with C = B it is twice the magnetic energy
    const vec& CX = cX ? *cX : bX;
    const vec& CY = cY ? *cY : bY;
    const vec& CZ = cZ ? *cZ : bZ;
    real s = 0.0;
    std::vector<real> bx(mL * mm), by(mm * mL), cx(mL * mm), cy(mm * mL);
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        int k = kid(ex, ey);
        clX(bX, ex, ey, bx.data()); clY(bY, ex, ey, by.data());
        clX(CX, ex, ey, cx.data()); clY(CY, ex, ey, cy.data());
        for (int qy = 0; qy < mL; ++qy)
          for (int qx = 0; qx < mL; ++qx) {
            real X = z2[qx], Y = z2[qy];
            s += Jdet * w2[qx] * w2[qy] *
                 (evX(bx.data(), X, Y) * evX(cx.data(), X, Y) + evY(by.data(), X, Y) * evY(cy.data(), X, Y));
          }
        const real* bz = &bZ[(size_t)k * mm * mm];
        const real* cz = &CZ[(size_t)k * mm * mm];
        for (int qy = 0; qy < mm; ++qy)
          for (int qx = 0; qx < mm; ++qx) {
            real X = zG[qx], Y = zG[qy];
            s += Jdet * wG[qx] * wG[qy] * evZ(bz, X, Y) * evZ(cz, X, Y);
          }
      }
    return s;
  }
};

// Host-array conversion of the C interface (values only; the tangent build
// exchanges tangents through or_set_tangent / or_get_tangent).
void to_host(double* out, const vec& v) {
  for (size_t i = 0; i < v.size(); ++i) out[i] = val(v[i]);
}
vec from_host(const double* p, size_t n) { return vec(p, p + n); }

}  // namespace

#include "mhd_oracle_stab.inc"

// ---------------------------------------------------------------------------
// C interface for the test-suite (ctypes)
// ---------------------------------------------------------------------------
extern "C" {

int or_rule(int kind, int r, double* x, double* w) {
  vec X, W;
  if (kind == 0) gauss_rule(r + 1, X, W);  // Gauss(r): r+1 points
  else gll_rule(r, X, W);                  // GLL(r): r+1 points
  to_host(x, X);
  to_host(w, W);
  return (int)X.size();
}

double or_lagrange(const double* nodes, int nn, int j, double x, int deriv) {
  vec v(nodes, nodes + nn);
  return val(deriv ? dlag(v, j, x) : lag(v, j, x));
}

double or_log_mean(double a, double b) { return val(log_mean(a, b)); }

void or_ec_flux(int d, const double* UL, const double* UR, double g, double* F) {
  vec l = from_host(UL, 5), r = from_host(UR, 5), f(5);
  ec_flux(d, l.data(), r.data(), g, f.data());
  to_host(F, f);
}
void or_llf_flux(int d, const double* Um, const double* Up, double g, double* F) {
  vec l = from_host(Um, 5), r = from_host(Up, 5), f(5);
  llf_flux(d, l.data(), r.data(), g, f.data());
  to_host(F, f);
}
void or_phys_flux(int d, const double* U, double g, double* F) {
  vec u = from_host(U, 5), f(5);
  phys_flux(d, u.data(), g, f.data());
  to_host(F, f);
}

void* or_create(int nx, int ny, double x0, double x1, double y0, double y1, int p, int m, double g) {
  if (nx < 1 || ny < 1 || p < 1 || m < 0 || m > p) return nullptr;
  Oracle* o = new Oracle();
  o->init(nx, ny, x0, x1, y0, y1, p, m, g);
  return o;
}
void or_destroy(void* h) { delete (Oracle*)h; }

// Threads of the OpenMP timing build (liboracle_omp.so): n > 0 sets the
// count; returns the count in force (1 in the serial builds).  The element
// loops it parallelises write disjoint data and every sum keeps its serial
// order, so the results equal the serial build's bit for bit.
int or_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void or_set_params(void* h, int oe_hydro, int oe_vel, int pp, int ar, double s_H, double s_M, double C_s,
                   double C_eta, double cfl, int max_halvings, int ec_faces) {
  Oracle* o = (Oracle*)h;
  const int frozen = o->prm.frozen, order = o->prm.strang_order;
  o->prm = Params{oe_hydro, oe_vel, pp, ar, s_H, s_M, C_s, C_eta, cfl, max_halvings, ec_faces, frozen, order};
}

// Ordering of the Strang composition: 0 H-M-H (default), 1 M-H-M (reading R20).
void or_set_strang_order(void* h, int order) { ((Oracle*)h)->prm.strang_order = order; }

// Tangent build: hold the stabilisation coefficients at their forward values
// (the linearisation that the library's adjoint differentiates).
void or_set_frozen(void* h, int frozen) { ((Oracle*)h)->prm.frozen = frozen; }

// Physical coordinates of the DG nodes [K][n2], of the W nodes
// [NY][NX] (GLL(m+1) nodes 0..m of each element) and of the B_z nodes [K][mm^2].
void or_coords(void* h, int which, double* X, double* Y) {
  Oracle* o = (Oracle*)h;
  for (int ey = 0; ey < o->ny; ++ey)
    for (int ex = 0; ex < o->nx; ++ex) {
      real xl = o->x0 + ex * o->hx, yl = o->y0 + ey * o->hy;
      int k = o->kid(ex, ey);
      if (which == 0) {
        for (int j = 0; j < o->n; ++j)
          for (int i = 0; i < o->n; ++i) {
            size_t q = (size_t)k * o->n2 + j * o->n + i;
            X[q] = val(xl + (1.0 + o->xp[i]) * o->hx / 2.0);
            Y[q] = val(yl + (1.0 + o->xp[j]) * o->hy / 2.0);
          }
      } else if (which == 1) {
        for (int b = 0; b < o->mm; ++b)
          for (int a = 0; a < o->mm; ++a) {
            size_t q = o->gidx(ex * o->mm + a, ey * o->mm + b);
            X[q] = val(xl + (1.0 + o->xL[a]) * o->hx / 2.0);
            Y[q] = val(yl + (1.0 + o->xL[b]) * o->hy / 2.0);
          }
      } else {
        for (int b = 0; b < o->mm; ++b)
          for (int a = 0; a < o->mm; ++a) {
            size_t q = (size_t)k * o->mm * o->mm + b * o->mm + a;
            X[q] = val(xl + (1.0 + o->xM[a]) * o->hx / 2.0);
            Y[q] = val(yl + (1.0 + o->xM[b]) * o->hy / 2.0);
          }
      }
    }
}

// In-plane field from a constant part plus the discrete rotated gradient of
// the nodal W-interpolant of a potential (reading R10): B = B0 + grad^perp A.
void or_b_from_potential(void* h, const double* Az, double Bx0, double By0, double* BxOut, double* ByOut) {
  Oracle* o = (Oracle*)h;
  vec A(Az, Az + (size_t)o->NX * o->NY);
  std::vector<real> c(o->mL * o->mL);
  for (int ey = 0; ey < o->ny; ++ey)
    for (int ex = 0; ex < o->nx; ++ex) {
      o->clW(A, ex, ey, c.data());
      for (int b = 0; b < o->mm; ++b)
        for (int a = 0; a < o->mm; ++a) {
          BxOut[o->gidx(ex * o->mm + a, ey * o->mm + b)] = val(Bx0 - (2.0 / o->hy) * o->evW(c.data(), o->xL[a], o->zG[b], 0, 1));
          ByOut[o->gidx(ex * o->mm + a, ey * o->mm + b)] = val(By0 + (2.0 / o->hx) * o->evW(c.data(), o->zG[a], o->xL[b], 1, 0));
        }
    }
}

void or_set_state(void* h, const double* U5, const double* bx, const double* by, const double* bz) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2;
  for (int c = 0; c < 5; ++c) o->U[c].assign(U5 + c * N, U5 + (c + 1) * N);
  size_t G = (size_t)o->NX * o->NY;
  o->Bx.assign(bx, bx + G); o->By.assign(by, by + G);
  o->Bz.assign(bz, bz + (size_t)o->K * o->mm * o->mm);
}

void or_get_state(void* h, double* U5, double* bx, double* by, double* bz) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2;
  for (int c = 0; c < 5; ++c) to_host(U5 + c * N, o->U[c]);
  to_host(bx, o->Bx);
  to_host(by, o->By);
  to_host(bz, o->Bz);
}

void or_hydro_rhs(void* h, const double* U5, double* L5) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2;
  vec S[5], L[5];
  for (int c = 0; c < 5; ++c) { S[c].assign(U5 + c * N, U5 + (c + 1) * N); L[c].assign(N, 0.0); }
  o->hydro_rhs(S, L);
  for (int c = 0; c < 5; ++c) to_host(L5 + c * N, L[c]);
}

// Magnetic residual on a primitive state: inputs rho, e, u (3 x N), B, etaK;
// outputs de, du (3 x N), dB; J and E (3 x G each) if non-null.
void or_mag_rhs(void* h, const double* rho, const double* e, const double* u, const double* bx, const double* by,
                const double* bz, const double* etaK, double* de, double* du, double* dbx, double* dby, double* dbz,
                double* Jo, double* Eo) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2, G = (size_t)o->NX * o->NY, Z = (size_t)o->K * o->mm * o->mm;
  Oracle::Mag Y, dY;
  Y.e.assign(e, e + N);
  for (int d = 0; d < 3; ++d) Y.u[d].assign(u + d * N, u + (d + 1) * N);
  Y.Bx.assign(bx, bx + G); Y.By.assign(by, by + G); Y.Bz.assign(bz, bz + Z);
  vec R(rho, rho + N), E(etaK, etaK + o->K);
  vec Jv[3], Ev[3];
  o->mag_rhs(R, E, Y, dY, Jv, Ev);
  to_host(de, dY.e);
  for (int d = 0; d < 3; ++d) to_host(du + d * N, dY.u[d]);
  to_host(dbx, dY.Bx);
  to_host(dby, dY.By);
  to_host(dbz, dY.Bz);
  if (Jo) for (int d = 0; d < 3; ++d) to_host(Jo + d * G, Jv[d]);
  if (Eo) for (int d = 0; d < 3; ++d) to_host(Eo + d * G, Ev[d]);
}

// (B, C)_B with the exact magnetic product.
double or_mag_product(void* h, const double* bx, const double* by, const double* bz, const double* cx,
                      const double* cy, const double* cz) {
  Oracle* o = (Oracle*)h;
  size_t G = (size_t)o->NX * o->NY, Z = (size_t)o->K * o->mm * o->mm;
  vec BX(bx, bx + G), BY(by, by + G), BZ(bz, bz + Z), CX(cx, cx + G), CY(cy, cy + G), CZ(cz, cz + Z);
  return val(o->mag_energy(BX, BY, BZ, &CX, &CY, &CZ));
}

// which = 0: hydro substep Phi_H^tau; which = 1: magnetic substep Phi_M^tau.
int or_substep(void* h, int which, double tau) {
  Oracle* o = (Oracle*)h;
  return which == 0 ? o->hydro_substep(tau) : o->run_mag(tau);
}

int or_strang_step(void* h, double dt, double* dt_taken, int* nrej) {
  Oracle* o = (Oracle*)h;
  real taken = 0.0;
  int st = o->strang_step(dt, &taken);
  if (dt_taken) *dt_taken = val(taken);
  if (nrej) *nrej = o->last_rejections;
  return st;
}

double or_cfl_dt(void* h) { return val(((Oracle*)h)->cfl_dt()); }
double or_div_metric(void* h) { return val(((Oracle*)h)->div_metric()); }

void or_get_eta(void* h, double* out) {
  Oracle* o = (Oracle*)h;
  to_host(out, o->eta);
}

// Element resistivity used by or_sample's E_h (normally the one the last
// magnetic substep computed); an input here, e.g. taken from another solver.
void or_set_eta(void* h, const double* in) {
  Oracle* o = (Oracle*)h;
  o->eta = from_host(in, (size_t)o->K);
}

// Diagnostics: [mass, mom_x, mom_y, mom_z, E_kin, E_int, E_mag, entropy S_h,
// div metric, max|B|, rho_min, p_min, eta_max].
void or_diagnostics(void* h, double* out) {
  Oracle* o = (Oracle*)h;
  real mass = 0, mom[3] = {0, 0, 0}, ekin = 0, eint = 0, S = 0, rmin = 1e300, pmin = 1e300, bmax = 0;
  for (int ey = 0; ey < o->ny; ++ey)
    for (int ex = 0; ex < o->nx; ++ex) {
      int k = o->kid(ex, ey);
      for (int j = 0; j < o->n; ++j)
        for (int i = 0; i < o->n; ++i) {
          real Ui[5]; o->node_state(o->U, k, i, j, Ui);
          real M = o->Jdet * o->wp[i] * o->wp[j];
          real pr = pressure(Ui, o->g);
          mass += M * Ui[0];
          for (int d = 0; d < 3; ++d) mom[d] += M * Ui[1 + d];
          ekin += M * 0.5 * (Ui[1] * Ui[1] + Ui[2] * Ui[2] + Ui[3] * Ui[3]) / Ui[0];
          eint += M * pr / (o->g - 1.0);
          S += M * Ui[0] * (log(pr) - o->g * log(Ui[0]));
          rmin = std::min(rmin, Ui[0]); pmin = std::min(pmin, pr);
          real B[3]; o->B_at_dg(ex, ey, i, j, B);
          bmax = std::max(bmax, sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
        }
    }
  real emax = 0; for (int k = 0; k < o->K; ++k) emax = std::max(emax, o->eta[k]);
  const real r[13] = {mass, mom[0], mom[1], mom[2], ekin, eint, 0.5 * o->mag_energy(o->Bx, o->By, o->Bz),
                      S, o->div_metric(), bmax, rmin, pmin, emax};
  for (int i = 0; i < 13; ++i) out[i] = val(r[i]);
}

// Physical coordinates of the nq x nq Gauss-Legendre points of every element,
// [K][qy][qx] with K = ey*nx + ex (the layout of or_sample).
void or_quad_coords(void* h, int nq, double* X, double* Y) {
  Oracle* o = (Oracle*)h;
  vec zq, wq; gauss_rule(nq, zq, wq);
  size_t idx = 0;
  for (int ey = 0; ey < o->ny; ++ey)
    for (int ex = 0; ex < o->nx; ++ex)
      for (int qy = 0; qy < nq; ++qy)
        for (int qx = 0; qx < nq; ++qx, ++idx) {
          X[idx] = val(o->x0 + ex * o->hx + (1.0 + zq[qx]) * o->hx / 2.0);
          Y[idx] = val(o->y0 + ey * o->hy + (1.0 + zq[qy]) * o->hy / 2.0);
        }
}

// Initial out-of-plane field as the L2(K) projection onto V_h^m (Q^m in the
// GLL(m) nodal basis of §3.1.3) of data given at the nq x nq Gauss points of
// every element (layout of or_quad_coords).  The paper does not state its
// initial B_z; this projection is the reading under which its Table 1 is
// reproduced.  For each element the (m+1)^2 normal equations
//   sum_b c_b (phi_b, phi_a)_K = (f, phi_a)_K  for every basis function a
// are assembled with the nq-point tensor rule (exact for the mass when
// nq >= m+1) and solved by Gaussian elimination with partial pivoting.
void or_project_Bz(void* h, const double* fq, int nq) {
  Oracle* o = (Oracle*)h;
  vec zq, wq; gauss_rule(nq, zq, wq);
  const int mm = o->mm, nb = mm * mm;
  std::vector<real> A((size_t)nb * nb), r(nb), phi((size_t)nb * nq * nq);
  for (int b = 0; b < nb; ++b)  // basis function b = (bx, by) at every point
    for (int qy = 0; qy < nq; ++qy)
      for (int qx = 0; qx < nq; ++qx)
        phi[((size_t)b * nq + qy) * nq + qx] = lag(o->xM, b % mm, zq[qx]) * lag(o->xM, b / mm, zq[qy]);
  for (int k = 0; k < o->K; ++k) {
    const double* f = fq + (size_t)k * nq * nq;
    for (int a = 0; a < nb; ++a) {
      r[a] = 0.0;
      for (int b = 0; b < nb; ++b) A[(size_t)a * nb + b] = 0.0;
      for (int qy = 0; qy < nq; ++qy)
        for (int qx = 0; qx < nq; ++qx) {
          real w = o->Jdet * wq[qx] * wq[qy];
          real pa = phi[((size_t)a * nq + qy) * nq + qx];
          r[a] += w * f[qy * nq + qx] * pa;
          for (int b = 0; b < nb; ++b) A[(size_t)a * nb + b] += w * pa * phi[((size_t)b * nq + qy) * nq + qx];
        }
    }
    for (int col = 0; col < nb; ++col) {  // forward elimination
      int piv = col;
      for (int i = col + 1; i < nb; ++i)
        if (fabs(A[(size_t)i * nb + col]) > fabs(A[(size_t)piv * nb + col])) piv = i;
      if (piv != col) {
        for (int j = 0; j < nb; ++j) std::swap(A[(size_t)col * nb + j], A[(size_t)piv * nb + j]);
        std::swap(r[col], r[piv]);
      }
      for (int i = col + 1; i < nb; ++i) {
        real l = A[(size_t)i * nb + col] / A[(size_t)col * nb + col];
        for (int j = col; j < nb; ++j) A[(size_t)i * nb + j] -= l * A[(size_t)col * nb + j];
        r[i] -= l * r[col];
      }
    }
    for (int i = nb - 1; i >= 0; --i) {  // back substitution
      real sum = r[i];
      for (int j = i + 1; j < nb; ++j) sum -= A[(size_t)i * nb + j] * o->Bz[(size_t)k * nb + j];
      o->Bz[(size_t)k * nb + i] = sum / A[(size_t)i * nb + i];
    }
  }
}

// Sample a field at the nq x nq Gauss points of every element (for L2 errors).
// field: 0..4 conserved, 5..7 u, 8 p, 9..11 B, 12..14 E_h, 15..17 J_h
// (E_h with the element resistivity of the last magnetic substep).
void or_sample(void* h, int field, int nq, double* val_out, double* X, double* Y, double* W) {
  Oracle* o = (Oracle*)h;
  vec zq, wq; gauss_rule(nq, zq, wq);
  vec Jv[3], Ev[3];
  if (field >= 12) {
    o->compute_J(o->Bx, o->By, o->Bz, Jv[0], Jv[1], Jv[2]);
    if (field < 15) {
      Oracle::Mag Y0; o->cons_to_prim(Y0);
      o->compute_E(Y0.u, o->Bx, o->By, o->Bz, o->eta, Jv[0], Jv[1], Jv[2], Ev[0], Ev[1], Ev[2]);
    }
  }
  std::vector<real> c(std::max(o->n2, o->mL * o->mL)), c2(o->n2);
  size_t idx = 0;
  for (int ey = 0; ey < o->ny; ++ey)
    for (int ex = 0; ex < o->nx; ++ex) {
      int k = o->kid(ex, ey);
      for (int qy = 0; qy < nq; ++qy)
        for (int qx = 0; qx < nq; ++qx, ++idx) {
          real xr = zq[qx], yr = zq[qy];
          X[idx] = val(o->x0 + ex * o->hx + (1.0 + xr) * o->hx / 2.0);
          Y[idx] = val(o->y0 + ey * o->hy + (1.0 + yr) * o->hy / 2.0);
          W[idx] = val(o->Jdet * wq[qx] * wq[qy]);
          real v = 0.0;
          if (field <= 4) {
            v = o->evDG(&o->U[field][(size_t)k * o->n2], xr, yr);
          } else if (field <= 7) {
            for (int q = 0; q < o->n2; ++q) c2[q] = o->U[field - 4][(size_t)k * o->n2 + q] / o->U[0][(size_t)k * o->n2 + q];
            v = o->evDG(c2.data(), xr, yr);
          } else if (field == 8) {
            for (int q = 0; q < o->n2; ++q) {
              real Ui[5]; for (int cc = 0; cc < 5; ++cc) Ui[cc] = o->U[cc][(size_t)k * o->n2 + q];
              c2[q] = pressure(Ui, o->g);
            }
            v = o->evDG(c2.data(), xr, yr);
          } else if (field == 9) { o->clX(o->Bx, ex, ey, c.data()); v = o->evX(c.data(), xr, yr); }
          else if (field == 10) { o->clY(o->By, ex, ey, c.data()); v = o->evY(c.data(), xr, yr); }
          else if (field == 11) { v = o->evZ(&o->Bz[(size_t)k * o->mm * o->mm], xr, yr); }
          else {
            const vec* F = field < 15 ? Ev : Jv;
            int comp = (field - 12) % 3;
            if (comp == 0) { o->clY(F[0], ex, ey, c.data()); v = o->evY(c.data(), xr, yr); }
            else if (comp == 1) { o->clX(F[1], ex, ey, c.data()); v = o->evX(c.data(), xr, yr); }
            else { o->clW(F[2], ex, ey, c.data()); v = o->evW(c.data(), xr, yr); }
          }
          val_out[idx] = val(v);
        }
    }
}

}  // extern "C"

#ifdef ORACLE_TANGENT
// ---------------------------------------------------------------------------
// Tangent interface (liboracle_tangent.so only): directional derivatives of the
// oracle's maps by forward-mode dual numbers.  The test-suite uses them as the
// exact tangent J dx against which the adjoint's J^T lam is checked.
// ---------------------------------------------------------------------------
namespace {
void seed(vec& v, const double* d) {
  for (size_t i = 0; i < v.size(); ++i) v[i].d = d ? d[i] : 0.0;
}
void tangent_out(double* out, const vec& v) {
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].d;
}
}  // namespace

extern "C" {

// Tangent parts of the current state (values unchanged).
void or_set_tangent(void* h, const double* dU5, const double* dbx, const double* dby, const double* dbz) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2;
  for (int c = 0; c < 5; ++c) seed(o->U[c], dU5 + c * N);
  seed(o->Bx, dbx); seed(o->By, dby); seed(o->Bz, dbz);
}

void or_get_tangent(void* h, double* dU5, double* dbx, double* dby, double* dbz) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2;
  for (int c = 0; c < 5; ++c) tangent_out(dU5 + c * N, o->U[c]);
  tangent_out(dbx, o->Bx); tangent_out(dby, o->By); tangent_out(dbz, o->Bz);
}

// L = L_E(U) and its tangent dL = L_E'(U) dU.
void or_hydro_rhs_tangent(void* h, const double* U5, const double* dU5, double* L5, double* dL5) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2;
  vec S[5], L[5];
  for (int c = 0; c < 5; ++c) {
    S[c] = from_host(U5 + c * N, N);
    seed(S[c], dU5 + c * N);
    L[c].assign(N, 0.0);
  }
  o->hydro_rhs(S, L);
  for (int c = 0; c < 5; ++c) { to_host(L5 + c * N, L[c]); tangent_out(dL5 + c * N, L[c]); }
}

// Magnetic residual (de, du, dB) of (rho, e, u, B) at fixed eta and its tangent
// for the input tangents (t_*); outputs out[0..4] = de, du, dBx, dBy, dBz and
// tout[0..4] their tangents.
void or_mag_rhs_tangent(void* h, const double* rho, const double* t_rho, const double* e, const double* t_e,
                        const double* u, const double* t_u, const double* bx, const double* t_bx,
                        const double* by, const double* t_by, const double* bz, const double* t_bz,
                        const double* etaK, double* de, double* du, double* dbx, double* dby, double* dbz,
                        double* t_de, double* t_du, double* t_dbx, double* t_dby, double* t_dbz) {
  Oracle* o = (Oracle*)h;
  size_t N = (size_t)o->K * o->n2, G = (size_t)o->NX * o->NY, Z = (size_t)o->K * o->mm * o->mm;
  Oracle::Mag Y, dY;
  Y.e = from_host(e, N); seed(Y.e, t_e);
  for (int d = 0; d < 3; ++d) { Y.u[d] = from_host(u + d * N, N); seed(Y.u[d], t_u + d * N); }
  Y.Bx = from_host(bx, G); seed(Y.Bx, t_bx);
  Y.By = from_host(by, G); seed(Y.By, t_by);
  Y.Bz = from_host(bz, Z); seed(Y.Bz, t_bz);
  vec R = from_host(rho, N), E = from_host(etaK, o->K);
  seed(R, t_rho);
  o->mag_rhs(R, E, Y, dY);
  to_host(de, dY.e); tangent_out(t_de, dY.e);
  for (int d = 0; d < 3; ++d) { to_host(du + d * N, dY.u[d]); tangent_out(t_du + d * N, dY.u[d]); }
  to_host(dbx, dY.Bx); tangent_out(t_dbx, dY.Bx);
  to_host(dby, dY.By); tangent_out(t_dby, dY.By);
  to_host(dbz, dY.Bz); tangent_out(t_dbz, dY.Bz);
}

}  // extern "C"
#endif
