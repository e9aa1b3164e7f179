// Adjoint (vector-Jacobian product) of the hydro residual L_E (§3.2.1,
// eq. euler-nodal-index) and the pointwise pieces of the adjoint Strang step.
//
// Given nu (5 x N) the kernels return (dL_E/dU)^T nu: the transposed flux
// differencing with the Jacobians of the entropy-conservative two-point flux
// (eq. euler-chandrashekar-flux) and of the LLF interface flux (eq.
// euler-lf-flux; at lambda = max(s-, s+) the side that attains the maximum
// carries the derivative).  Reverse mode is written out by hand below, one
// adjoint statement per forward statement in reverse order.  Only the
// unstabilised residual is differentiated: the OE map and the limiter are
// outside the adjoint (the driver flags them when they are on).
#include "mhd_internal.cuh"

namespace mhd {

struct Prim {
  double r, u[3], p, u2;
};

__device__ __forceinline__ Prim prim_of(const double U[5], double g) {
  Prim q;
  q.r = U[0];
  const double ir = 1.0 / U[0];
  q.u[0] = U[1] * ir; q.u[1] = U[2] * ir; q.u[2] = U[3] * ir;
  q.u2 = q.u[0] * q.u[0] + q.u[1] * q.u[1] + q.u[2] * q.u[2];
  q.p = (g - 1.0) * (U[4] - 0.5 * U[0] * q.u2);
  return q;
}

// Adjoint of (rho, m, E) -> (rho, u, p): given gr (direct rho part), gu, gp,
// accumulate into out (conservative adjoint).
__device__ __forceinline__ void prim_adjoint(const Prim& q, double g, double gr, const double gu[3], double gp,
                                             double out[5]) {
  const double ir = 1.0 / q.r;
  // p = (g-1)(E - |m|^2/(2 rho))
  out[4] += (g - 1.0) * gp;
  double dr = gr + (g - 1.0) * gp * 0.5 * q.u2;
  for (int c = 0; c < 3; ++c) {
    out[1 + c] += gu[c] * ir - (g - 1.0) * gp * q.u[c];
    dr -= gu[c] * q.u[c] * ir;  // u = m / rho
  }
  out[0] += dr;
}

// Log-mean factor F(aL, aR) with a_log = (aL + aR)/(2F) (reading R1) and its
// partial derivatives dF/daL, dF/daR.
__device__ __forceinline__ double logmean_F(double aL, double aR, double* dFL, double* dFR) {
  const double s = aL + aR, d = aL - aR;
  const double f = d / s, u = f * f;
  const double dfL = 2.0 * aR / (s * s), dfR = -2.0 * aL / (s * s);
  if (u < 1e-4) {
    const double F = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0;
    const double dFdf = 2.0 * f * (1.0 / 3.0 + 2.0 * u / 5.0 + 3.0 * u * u / 7.0);
    *dFL = dFdf * dfL;
    *dFR = dFdf * dfR;
    return F;
  }
  const double lz = log(aL / aR);
  const double F = lz / (2.0 * f);
  *dFL = (1.0 / aL) / (2.0 * f) - lz / (2.0 * f * f) * dfL;
  *dFR = (-1.0 / aR) / (2.0 * f) - lz / (2.0 * f * f) * dfR;
  return F;
}

// dL += (dF_ec/dUL)^T gF, dR += (dF_ec/dUR)^T gF (direction d).
__device__ void ec_flux_vjp(int d, const double UL[5], const double UR[5], double g, const double gF[5], double dL[5],
                            double dR[5]) {
  const Prim L = prim_of(UL, g), R = prim_of(UR, g);
  const double bL = L.r / (2.0 * L.p), bR = R.r / (2.0 * R.p);
  double dFrL, dFrR, dFbL, dFbR;
  const double Fr = logmean_F(L.r, R.r, &dFrL, &dFrR);
  const double Fb = logmean_F(bL, bR, &dFbL, &dFbR);
  const double sr = L.r + R.r, sb = bL + bR;
  const double rlog = 0.5 * sr / Fr;
  double ua[3];
  for (int c = 0; c < 3; ++c) ua[c] = 0.5 * (L.u[c] + R.u[c]);
  const double ig1 = 1.0 / (g - 1.0);
  const double hhat = (Fb * ig1 + Fr) / sb - 0.25 * (L.u2 + R.u2) + ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2];
  const double ud = ua[d];
  const double f0 = rlog * ud;
  // reverse sweep
  const double gf0 = gF[0] + gF[1] * ua[0] + gF[2] * ua[1] + gF[3] * ua[2] + gF[4] * hhat;
  double gua[3] = {gF[1] * f0, gF[2] * f0, gF[3] * f0};
  gua[d] += gf0 * rlog;
  const double gphat = d == 0 ? gF[1] : gF[2];
  const double ghhat = gF[4] * f0;
  const double grlog = gf0 * ud;
  double gFb = ghhat * ig1 / sb, gFr = ghhat / sb;
  double gsb = -ghhat * (Fb * ig1 + Fr) / (sb * sb);
  const double gu2a = -0.5 * ghhat;  // u2a = (|uL|^2 + |uR|^2)/2
  for (int c = 0; c < 3; ++c) gua[c] += 2.0 * ua[c] * ghhat;
  double gsr = 0.5 * gphat / sb;  // phat = sr / (2 sb)
  gsb -= 0.5 * gphat * sr / (sb * sb);
  gsr += 0.5 * grlog / Fr;  // rlog = sr / (2 Fr)
  gFr -= 0.5 * grlog * sr / (Fr * Fr);
  double guL[3], guR[3];
  for (int c = 0; c < 3; ++c) {
    guL[c] = 0.5 * gua[c] + gu2a * L.u[c];
    guR[c] = 0.5 * gua[c] + gu2a * R.u[c];
  }
  const double grL = gsr + gFr * dFrL, grR = gsr + gFr * dFrR;
  const double gbL = gsb + gFb * dFbL, gbR = gsb + gFb * dFbR;
  // beta = rho / (2 p)
  prim_adjoint(L, g, grL + gbL / (2.0 * L.p), guL, -gbL * bL / L.p, dL);
  prim_adjoint(R, g, grR + gbR / (2.0 * R.p), guR, -gbR * bR / R.p, dR);
}

// out += (dF_d/dU)^T h for the physical flux F_d.
__device__ void phys_flux_vjp(int d, const double U[5], double g, const double h[5], double out[5]) {
  const Prim q = prim_of(U, g);
  const double ud = q.u[d];
  double gu[3] = {0.0, 0.0, 0.0};
  double gp = 0.0;
  out[1 + d] += h[0];
  out[1] += h[1] * ud; gu[d] += h[1] * U[1]; if (d == 0) gp += h[1];
  out[2] += h[2] * ud; gu[d] += h[2] * U[2]; if (d == 1) gp += h[2];
  out[3] += h[3] * ud; gu[d] += h[3] * U[3];
  out[4] += h[4] * ud; gp += h[4] * ud; gu[d] += h[4] * (U[4] + q.p);
  prim_adjoint(q, g, 0.0, gu, gp, out);
}

// out += gs * ds/dU, s = |u_d| + c, c = sqrt(g p / rho).
__device__ void speed_vjp(int d, const double U[5], double g, double gs, double out[5]) {
  const Prim q = prim_of(U, g);
  const double c = sqrt(g * q.p / q.r);
  double gu[3] = {0.0, 0.0, 0.0};
  gu[d] = q.u[d] >= 0.0 ? gs : -gs;
  const double gp = gs * g / (2.0 * c * q.r);
  const double gr = -gs * c / (2.0 * q.r);
  prim_adjoint(q, g, gr, gu, gp, out);
}

__device__ void llf_flux_vjp(int d, const double Um[5], const double Up[5], double g, const double gF[5],
                             double dm[5], double dp[5]) {
  double h[5];
  for (int c = 0; c < 5; ++c) h[c] = 0.5 * gF[c];
  phys_flux_vjp(d, Um, g, h, dm);
  phys_flux_vjp(d, Up, g, h, dp);
  const Prim qm = prim_of(Um, g), qp = prim_of(Up, g);
  const double sm = fabs(qm.u[d]) + sqrt(g * qm.p / qm.r);
  const double sp = fabs(qp.u[d]) + sqrt(g * qp.p / qp.r);
  const double lam = fmax(sm, sp);
  double glam = 0.0;
  for (int c = 0; c < 5; ++c) {
    dp[c] -= 0.5 * lam * gF[c];
    dm[c] += 0.5 * lam * gF[c];
    glam -= 0.5 * (Up[c] - Um[c]) * gF[c];
  }
  if (sm >= sp) speed_vjp(d, Um, g, glam, dm);
  else speed_vjp(d, Up, g, glam, dp);
}

// Face part: for every face node, the adjoint of F* seen by the two end nodes;
// FA[dir][side][c][K][n], side 0 = minus trace (end node of the lower element),
// side 1 = plus trace (node 0 of element K).
template <int P>
__global__ void k_adj_face(const double* __restrict__ S, const double* __restrict__ nu, double* __restrict__ FA,
                           Mesh M, const Tab* __restrict__ T) {
  constexpr int n = P + 1, n2 = n * n;
  const size_t N = (size_t)M.K * n2, nf = (size_t)M.K * n;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nf) return;
  const int d = t >= nf;
  const size_t r = d ? t - nf : t;
  const int k = (int)(r / n), j = (int)(r % n);
  const int ex = k % M.nx, ey = k / M.nx;
  int km, qm, qp;
  if (d == 0) { km = ey * M.nx + wrap(ex - 1, M.nx); qm = j * n + P; qp = j * n; }
  else { km = wrap(ey - 1, M.ny) * M.nx + ex; qm = P * n + j; qp = j; }
  double Um[5], Up[5], gF[5], dm[5] = {0, 0, 0, 0, 0}, dp[5] = {0, 0, 0, 0, 0};
  const double f = 2.0 / ((d == 0 ? M.hx : M.hy) * T->wp[0]);
  for (int c = 0; c < 5; ++c) {
    Um[c] = S[c * N + (size_t)km * n2 + qm];
    Up[c] = S[c * N + (size_t)k * n2 + qp];
    gF[c] = f * (nu[c * N + (size_t)k * n2 + qp] - nu[c * N + (size_t)km * n2 + qm]);
  }
  llf_flux_vjp(d, Um, Up, M.g, gF, dm, dp);
  double* base = FA + (size_t)d * 2 * 5 * nf;
  for (int c = 0; c < 5; ++c) {
    base[(0 * 5 + c) * nf + r] = dm[c];
    base[(1 * 5 + c) * nf + r] = dp[c];
  }
}

// Volume part and assembly: one thread per element.  out = (dL_E/dU)^T nu.
template <int P>
__global__ void k_adj_vol(const double* __restrict__ S, const double* __restrict__ nu, const double* __restrict__ FA,
                          double* __restrict__ out, Mesh M, const Tab* __restrict__ T) {
  constexpr int n = P + 1, n2 = n * n;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.K) return;
  const size_t N = (size_t)M.K * n2, nf = (size_t)M.K * n;
  const int ex = k % M.nx, ey = k / M.nx;
  double lam[5][n2];
  for (int c = 0; c < 5; ++c)
    for (int q = 0; q < n2; ++q) lam[c][q] = 0.0;
  for (int dir = 0; dir < 2; ++dir) {
    const double cs = -4.0 / (dir == 0 ? M.hx : M.hy);
    for (int line = 0; line < n; ++line)
      for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
          const int qa = dir == 0 ? line * n + a : a * n + line;
          const int qb = dir == 0 ? line * n + b : b * n + line;
          double Ua[5], Ub[5], gF[5], da[5] = {0, 0, 0, 0, 0}, db[5] = {0, 0, 0, 0, 0};
          for (int c = 0; c < 5; ++c) {
            Ua[c] = S[c * N + (size_t)k * n2 + qa];
            Ub[c] = S[c * N + (size_t)k * n2 + qb];
            gF[c] = cs * (T->D[a][b] * nu[c * N + (size_t)k * n2 + qa] + T->D[b][a] * nu[c * N + (size_t)k * n2 + qb]);
          }
          ec_flux_vjp(dir, Ua, Ub, M.g, gF, da, db);
          for (int c = 0; c < 5; ++c) { lam[c][qa] += da[c]; lam[c][qb] += db[c]; }
        }
  }
  // interface parts: node 0 of a line is the plus trace of the lower face of this
  // element, node p the minus trace of the lower face of the upper neighbour
  const int kE = ey * M.nx + wrap(ex + 1, M.nx), kN = wrap(ey + 1, M.ny) * M.nx + ex;
  const double* FAx = FA;
  const double* FAy = FA + 2 * 5 * nf;
  for (int j = 0; j < n; ++j)
    for (int c = 0; c < 5; ++c) {
      lam[c][j * n + 0] += FAx[(1 * 5 + c) * nf + (size_t)k * n + j];
      lam[c][j * n + P] += FAx[(0 * 5 + c) * nf + (size_t)kE * n + j];
      lam[c][0 * n + j] += FAy[(1 * 5 + c) * nf + (size_t)k * n + j];
      lam[c][P * n + j] += FAy[(0 * 5 + c) * nf + (size_t)kN * n + j];
    }
  for (int c = 0; c < 5; ++c)
    for (int q = 0; q < n2; ++q) out[c * N + (size_t)k * n2 + q] = lam[c][q];
}

void hydro_rhs_vjp(int p, const double* S, const double* nu, double* FA, double* out, const Mesh& M, const Tab* T,
                   cudaStream_t st) {
  const size_t nf = (size_t)M.K * (p + 1);
  const unsigned bf = (unsigned)((2 * nf + 127) / 128), bv = (unsigned)((M.K + 63) / 64);
  switch (p) {
    case 1: k_adj_face<1><<<bf, 128, 0, st>>>(S, nu, FA, M, T); k_adj_vol<1><<<bv, 64, 0, st>>>(S, nu, FA, out, M, T); break;
    case 2: k_adj_face<2><<<bf, 128, 0, st>>>(S, nu, FA, M, T); k_adj_vol<2><<<bv, 64, 0, st>>>(S, nu, FA, out, M, T); break;
    case 3: k_adj_face<3><<<bf, 128, 0, st>>>(S, nu, FA, M, T); k_adj_vol<3><<<bv, 64, 0, st>>>(S, nu, FA, out, M, T); break;
    case 4: k_adj_face<4><<<bf, 128, 0, st>>>(S, nu, FA, M, T); k_adj_vol<4><<<bv, 64, 0, st>>>(S, nu, FA, out, M, T); break;
  }
}

// ---- pointwise adjoint pieces -------------------------------------------------
// y = a x + b y over n entries.
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], b * y[i]);
}

void axpby(double a, const double* x, double b, double* y, size_t n, cudaStream_t st) {
  k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, x, b, y, n);
}

// Adjoint of (e, u) -> (m, E) with frozen rho: m = rho u, E = rho e + rho|u|^2/2.
// In: lamU (5 x N: rho, m, E adjoints), Y (e, u).  Out: lamY (e, u adjoints),
// lamR += direct rho part.
__global__ void k_adj_prim_to_cons(const double* __restrict__ U, const double* __restrict__ Y,
                                   const double* __restrict__ lamU, double* __restrict__ lamY,
                                   double* __restrict__ lamR, size_t N) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const double rho = U[q], e = Y[q];
  const double u[3] = {Y[N + q], Y[2 * N + q], Y[3 * N + q]};
  const double lE = lamU[4 * N + q];
  double lr = lamU[q] + lE * (e + 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  lamY[q] = rho * lE;
  for (int c = 0; c < 3; ++c) {
    const double lm = lamU[(1 + c) * N + q];
    lamY[(1 + c) * N + q] = rho * lm + rho * u[c] * lE;
    lr += u[c] * lm;
  }
  lamR[q] = lr;
}

// Adjoint of (rho, m, E) -> (e, u): u = m/rho, e = E/rho - |m|^2/(2 rho^2).
// In: lamY (e, u), lamR (rho, accumulated).  Out: lamU (rho, m, E).
__global__ void k_adj_cons_to_prim(const double* __restrict__ U, const double* __restrict__ lamY,
                                   const double* __restrict__ lamR, double* __restrict__ lamU, size_t N) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const double rho = U[q], ir = 1.0 / rho, E = U[4 * N + q];
  const double m[3] = {U[N + q], U[2 * N + q], U[3 * N + q]};
  const double m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
  const double le = lamY[q];
  double lr = lamR[q] + le * (-E * ir * ir + m2 * ir * ir * ir);
  for (int c = 0; c < 3; ++c) {
    const double lu = lamY[(1 + c) * N + q];
    lamU[(1 + c) * N + q] = lu * ir - le * m[c] * ir * ir;
    lr -= lu * m[c] * ir * ir;
  }
  lamU[4 * N + q] = le * ir;
  lamU[q] = lr;
}

void adj_prim_to_cons(const double* U, const double* Y, const double* lamU, double* lamY, double* lamR, size_t N,
                      cudaStream_t st) {
  k_adj_prim_to_cons<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(U, Y, lamU, lamY, lamR, N);
}
void adj_cons_to_prim(const double* U, const double* lamY, const double* lamR, double* lamU, size_t N,
                      cudaStream_t st) {
  k_adj_cons_to_prim<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(U, lamY, lamR, lamU, N);
}

}  // namespace mhd
