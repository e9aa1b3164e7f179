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
// outside this residual adjoint (the step adjoint reports them in its flags).
#include "mhd_internal.cuh"

namespace mhd {

struct Prim {
  double r, u[3], p, u2;
};

__device__ __forceinline__ Prim prim_of(const double U[5], double g) {
  Prim q;
  q.r = U[0];
  const double ir = rcp(U[0]);
  q.u[0] = U[1] * ir; q.u[1] = U[2] * ir; q.u[2] = U[3] * ir;
  q.u2 = q.u[0] * q.u[0] + q.u[1] * q.u[1] + q.u[2] * q.u[2];
  q.p = (g - 1.0) * (U[4] - 0.5 * U[0] * q.u2);
  return q;
}

// Adjoint of (rho, m, E) -> (rho, u, p): given gr (direct rho part), gu, gp,
// accumulate into out (conservative adjoint).
__device__ __forceinline__ void prim_adjoint(const Prim& q, double g, double gr, const double gu[3], double gp,
                                             double out[5]) {
  const double ir = rcp(q.r);
  // p = (g-1)(E - |m|^2/(2 rho))
  out[4] += (g - 1.0) * gp;
  double dr = gr + (g - 1.0) * gp * 0.5 * q.u2;
  for (int c = 0; c < 3; ++c) {
    out[1 + c] += gu[c] * ir - (g - 1.0) * gp * q.u[c];
    dr -= gu[c] * q.u[c] * ir;  // u = m / rho
  }
  out[0] += dr;
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
  const double f = 2.0 * (d == 0 ? M.ihx : M.ihy) * (0.5 * P * (P + 1));  // 2 / (h w_0), w_0 = 2 / (p (p+1))
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

// Pair tables of the forward volume kernel (hydro.cu): pair w of a line is
// (c_pair_a[w], c_pair_b[w]) with w = b (b - 1) / 2 + a.
__constant__ unsigned char c_apair_a[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
__constant__ unsigned char c_apair_b[10] = {1, 2, 2, 3, 3, 3, 4, 4, 4, 4};

template <int P>
struct ACfg {
  static constexpr int n = P + 1, n2 = n * n;
  static constexpr int npairs = P * n2;        // unique pairs per element (both directions)
  static constexpr int npl = n * (n - 1) / 2;  // pairs per line
  static constexpr int EB = P == 1 ? 32 : (P == 2 ? 16 : (P == 3 ? 8 : 4));
  static constexpr int threads = EB * n2;
};

// F(f) = atanh(f)/f with a_log = (aL + aR)/(2F), f = (aL - aR)/(aL + aR), and
// F'(f): the Taylor series sum_k f^2k/(2k+1) for f^2 < 1e-2 (eight terms,
// truncation below 1e-17), otherwise from per-node logarithms, lz = log aL -
// log aR = 2 atanh(f): F = lz/(2f), F' = (1/(1 - f^2) - F)/f.
__device__ __forceinline__ double logmean_FdF(double f, double lz, double* dF, double* iF) {
  const double u = f * f;
  if (__double_as_longlong(u) < __double_as_longlong(1e-2)) {  // u >= 0: integer compare of the bit patterns
    const double c[8] = {1.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 7.0, 1.0 / 9.0, 1.0 / 11.0, 1.0 / 13.0, 1.0 / 15.0};
    double F = c[7], G = 7.0 * 2.0 * c[7];
#pragma unroll
    for (int k = 6; k >= 1; --k) {
      F = fma(F, u, c[k]);
      G = fma(G, u, 2.0 * k * c[k]);
    }
    F = fma(F, u, c[0]);
    *dF = G * f;
    *iF = rcp(F);
    return F;
  }
  const double i2f = rcp(2.0 * f);
  const double F = lz * i2f;
  *dF = (rcp(1.0 - u) - F) * (2.0 * i2f);
  *iF = (2.0 * f) / lz;
  return F;
}

// Whether node value x of an element can put a pair of the element on the
// logarithm branch of logmean_FdF (f^2 >= 1e-2, i.e. a ratio of at least
// 1.1/0.9 = 1.2222) against the element's reference node value r: two nodes
// whose bit patterns are within 0.099 2^52 of r's have a ratio below
// exp(0.198) = 1.2190 (each ulp is a relative step of at most 2^-52), so only
// blocks with a node further away need the per-node logarithms.  Integer
// pipe only; non-positive or NaN values give huge differences.
__device__ __forceinline__ bool adj_far_from_reference(double x, double r) {
  const long long d = __double_as_longlong(x) - __double_as_longlong(r);
  constexpr long long lim = 445856363109670LL;  // 0.099 * 2^52, rounded down
  return d >= lim || d <= -lim;
}

// Volume part and assembly: EB elements x (p+1)^2 threads, p pairs per
// thread as in the forward kernel.  Each pair's reverse sweep yields the
// adjoints of (rho, u, beta) of its two nodes (shared memory); each node then
// sums its 2p pair contributions, converts them to the conservative adjoint
// once, and adds the interface contributions of k_adj_face.
template <int P>
__global__ void __launch_bounds__(ACfg<P>::threads) k_adj_vol(const double* __restrict__ S,
                                                              const double* __restrict__ nu,
                                                              const double* __restrict__ FA,
                                                              double* __restrict__ out, Mesh M,
                                                              const Tab* __restrict__ T) {
  using C = ACfg<P>;
  constexpr int n = C::n, n2 = C::n2, EB = C::EB, NP = C::npairs, NPL = C::npl;
  __shared__ double sp[8][EB * n2];   // rho, ux, uy, uz, beta, |u|^2, log rho, log beta
  __shared__ double sn[5][EB * n2];   // nu
  __shared__ double sg[10][EB * NP];  // pair outputs: (g_rho, g_u, g_beta) of node a, then of node b
  const size_t N = (size_t)M.K * n2;
  const int tid = threadIdx.x;
  const int el = tid / n2, q = tid % n2;
  const int k = blockIdx.x * EB + el;
  const bool valid = k < M.K;
  const int kk = valid ? k : M.K - 1;
  const size_t gi = (size_t)kk * n2 + q;
  const double g = M.g, ig1 = M.ig1;
  double r0, u0[3], b0, u20;
  {
    double Us[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      Us[c] = S[c * N + gi];
      sn[c][tid] = nu[c * N + gi];
    }
    const double ir = rcp(Us[0]);
    u0[0] = Us[1] * ir; u0[1] = Us[2] * ir; u0[2] = Us[3] * ir;
    u20 = fma(u0[0], u0[0], fma(u0[1], u0[1], u0[2] * u0[2]));
    const double pr = (g - 1.0) * fma(-0.5 * Us[0], u20, Us[4]);
    r0 = Us[0];
    b0 = 0.5 * Us[0] * rcp(pr);
    sp[0][tid] = r0; sp[1][tid] = u0[0]; sp[2][tid] = u0[1]; sp[3][tid] = u0[2];
    sp[4][tid] = b0; sp[5][tid] = u20;
  }
  __syncthreads();
  // per-node logarithms for the whole block, only if some element of it has a
  // node far enough from its first node for a pair to take the log branch
  const bool far = adj_far_from_reference(r0, sp[0][el * n2]) || adj_far_from_reference(b0, sp[4][el * n2]);
  const bool have_logs = __syncthreads_or(far) != 0;
  if (have_logs) {
    sp[6][tid] = log(r0);
    sp[7][tid] = log(b0);
    __syncthreads();
  }
  const double cs[2] = {-4.0 * M.ihx, -4.0 * M.ihy};
#pragma unroll
  for (int s = 0; s < P; ++s) {
    const int pidx = q + s * n2;
    const int d = pidx >= NP / 2;
    const int r = pidx - d * (NP / 2);
    const int line = r / NPL, w = r % NPL;
    const int a = c_apair_a[w], b = c_apair_b[w];
    const int qa = el * n2 + (d == 0 ? line * n + a : a * n + line);
    const int qb = el * n2 + (d == 0 ? line * n + b : b * n + line);
    // adjoint of the pair flux: it enters L_a with -(4/h) D_ab and L_b with -(4/h) D_ba
    const double Dab = cs[d] * T->D[a][b], Dba = cs[d] * T->D[b][a];
    double gF[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) gF[c] = fma(Dab, sn[c][qa], Dba * sn[c][qb]);
    const double rL = sp[0][qa], rR = sp[0][qb], bL = sp[4][qa], bR = sp[4][qb];
    const double sr = rL + rR, sb = bL + bR;
    const double isr = rcp(sr), isb = rcp(sb);
    const double fr = (rL - rR) * isr, fb = (bL - bR) * isb;
    double dFr, dFb, iFr, iFb;
    const double lzr = have_logs ? sp[6][qa] - sp[6][qb] : 0.0, lzb = have_logs ? sp[7][qa] - sp[7][qb] : 0.0;
    const double Fr = logmean_FdF(fr, lzr, &dFr, &iFr);
    const double Fb = logmean_FdF(fb, lzb, &dFb, &iFb);
    const double rlog = 0.5 * sr * iFr;
    double ua[3];
    ua[0] = 0.5 * (sp[1][qa] + sp[1][qb]);
    ua[1] = 0.5 * (sp[2][qa] + sp[2][qb]);
    ua[2] = 0.5 * (sp[3][qa] + sp[3][qb]);
    const double u2a = 0.5 * (sp[5][qa] + sp[5][qb]);
    const double au2 = fma(ua[0], ua[0], fma(ua[1], ua[1], ua[2] * ua[2]));
    const double hnum = fma(Fb, ig1, Fr);
    const double hhat = fma(hnum, isb, fma(-0.5, u2a, au2));
    const double ud = d == 0 ? ua[0] : ua[1];
    const double f0 = rlog * ud;
    // reverse sweep
    const double gf0 = fma(gF[1], ua[0], fma(gF[2], ua[1], fma(gF[3], ua[2], fma(gF[4], hhat, gF[0]))));
    double gua[3] = {gF[1] * f0, gF[2] * f0, gF[3] * f0};
    gua[d] = fma(gf0, rlog, gua[d]);
    const double gphat = gF[1 + d];
    const double ghhat = gF[4] * f0;
    const double grlog = gf0 * ud;
    const double gFb = ghhat * ig1 * isb;
    double gFr = ghhat * isb;
    double gsb = -ghhat * hnum * isb * isb;
    const double gu2a = -0.5 * ghhat;
#pragma unroll
    for (int c = 0; c < 3; ++c) gua[c] = fma(2.0 * ua[c], ghhat, gua[c]);
    double gsr = 0.5 * gphat * isb;
    gsb -= 0.5 * gphat * sr * isb * isb;
    gsr = fma(0.5 * grlog, iFr, gsr);
    gFr -= grlog * rlog * iFr;
    const double gfr = gFr * dFr, gfb = gFb * dFb;
    const int o = el * NP + pidx;
    sg[0][o] = fma(gfr * (1.0 - fr), isr, gsr);
    sg[5][o] = fma(-gfr * (1.0 + fr), isr, gsr);
    sg[4][o] = fma(gfb * (1.0 - fb), isb, gsb);
    sg[9][o] = fma(-gfb * (1.0 + fb), isb, gsb);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sg[1 + c][o] = fma(gu2a, sp[1 + c][qa], 0.5 * gua[c]);
      sg[6 + c][o] = fma(gu2a, sp[1 + c][qb], 0.5 * gua[c]);
    }
  }
  __syncthreads();
  // gather the pair outputs of this node: x-pairs on row j, y-pairs on column i
  const int i = q % n, j = q / n;
  double gr = 0.0, gu[3] = {0.0, 0.0, 0.0}, gb = 0.0;
#pragma unroll
  for (int rr = 0; rr < n; ++rr) {
    if (rr == i) continue;
    const int o = el * NP + j * NPL + (i < rr ? rr * (rr - 1) / 2 + i : i * (i - 1) / 2 + rr);
    const int side = i < rr ? 0 : 5;
    gr += sg[side][o]; gu[0] += sg[side + 1][o]; gu[1] += sg[side + 2][o]; gu[2] += sg[side + 3][o];
    gb += sg[side + 4][o];
  }
#pragma unroll
  for (int rr = 0; rr < n; ++rr) {
    if (rr == j) continue;
    const int o = el * NP + NP / 2 + i * NPL + (j < rr ? rr * (rr - 1) / 2 + j : j * (j - 1) / 2 + rr);
    const int side = j < rr ? 0 : 5;
    gr += sg[side][o]; gu[0] += sg[side + 1][o]; gu[1] += sg[side + 2][o]; gu[2] += sg[side + 3][o];
    gb += sg[side + 4][o];
  }
  // (rho, u, beta) -> conservative: beta = rho/(2p), p = (g-1)(E - rho |u|^2/2)
  const double ir = rcp(r0);
  const double gp = -2.0 * gb * b0 * b0 * ir;  // dbeta/dp = -beta/p, 1/p = 2 beta/rho
  gr = fma(gb * b0, ir, gr);                  // dbeta/drho at fixed p = 1/(2p)
  double res[5];
  res[4] = (g - 1.0) * gp;
  double dr = fma(0.5 * u20, res[4], gr);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    res[1 + c] = fma(gu[c], ir, -res[4] * u0[c]);
    dr -= gu[c] * u0[c] * ir;
  }
  res[0] = dr;
  // interface parts: node 0 of a line is the plus trace of the element's lower
  // face, node p the minus trace of the lower face of the next element
  const size_t nf = (size_t)M.K * n;
  const int ex = kk % M.nx, ey = kk / M.nx;
  const double* FAx = FA;
  const double* FAy = FA + 2 * 5 * nf;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double v = res[c];
    if (i == 0) v += FAx[(5 + c) * nf + (size_t)kk * n + j];
    if (i == P) v += FAx[c * nf + (size_t)(ey * M.nx + wrap(ex + 1, M.nx)) * n + j];
    if (j == 0) v += FAy[(5 + c) * nf + (size_t)kk * n + i];
    if (j == P) v += FAy[c * nf + (size_t)(wrap(ey + 1, M.ny) * M.nx + ex) * n + i];
    if (valid) out[c * N + gi] = v;
  }
}

void hydro_rhs_vjp(int p, const double* S, const double* nu, double* FA, double* out, const Mesh& M, const Tab* T,
                   cudaStream_t st) {
  const size_t nf = (size_t)M.K * (p + 1);
  const unsigned bf = (unsigned)((2 * nf + 127) / 128);
#define MHD_ADJ_H(PP)                                                                                   \
  k_adj_face<PP><<<bf, 128, 0, st>>>(S, nu, FA, M, T);                                                 \
  k_adj_vol<PP><<<(unsigned)((M.K + ACfg<PP>::EB - 1) / ACfg<PP>::EB), ACfg<PP>::threads, 0, st>>>(S, nu, FA, \
                                                                                                    out, M, T)
  switch (p) {
    case 1: MHD_ADJ_H(1); break;
    case 2: MHD_ADJ_H(2); break;
    case 3: MHD_ADJ_H(3); break;
    case 4: MHD_ADJ_H(4); break;
  }
#undef MHD_ADJ_H
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
  const double rho = U[q], ir = rcp(rho), E = U[4 * N + q];
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
