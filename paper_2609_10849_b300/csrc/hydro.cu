// Hydro stage kernels: entropy-stable DGSEM residual (§3.2.1, eq.
// euler-nodal-index) fused with the SSP-RK(3,3) stage combination
// (eq. euler-ssprk33) and the raw-average admissibility check (§3.2.3).
//
// Work mapping (FP64-issue bound part: every warp lane carries FP64 work):
//   k_face  one thread per face node: LLF flux (eq. euler-lf-flux) on every
//           x- and y-face, stored once per face as 2 F*: Fs[c][K][n], indexed
//           by the element on the + side of the face.
//   k_vol   EB elements x (p+1)^2 threads per block; the p(p+1)^2 unique
//           entropy-conservative pairs of an element (eq.
//           euler-chandrashekar-flux) are spread p per thread and evaluated
//           once (the flux is symmetric), then gathered with D.  With
//           2 D_00 = -1/w_0 and 2 D_pp = 1/w_p (SBP, eq. euler-sbp) the
//           physical-flux diagonal cancels the physical part of the surface
//           term exactly, leaving only the numerical flux F* at the end nodes.
#include "mhd_internal.cuh"

namespace mhd {

template <int P, int EBv = vol_tile_eb(P, 0)>
struct HCfg {
  static constexpr int n = P + 1, n2 = n * n;
  static constexpr int npairs = P * n2;        // unique pairs per element
  static constexpr int npl = n * (n - 1) / 2;  // pairs per line
  static constexpr int EB = EBv;               // elements per CTA (autotuned variant)
  static constexpr int threads = EB * n2;
  // resident warps per SM: the pair and gather phases wait on shared-memory
  // loads and reciprocal seeds, which more warps hide.  40 at p = 1 and p = 3
  // (48 registers, no spills; shared memory allows 36 at p = 3 with 8 elements
  // per CTA), 32 at p = 2 and p = 4, where 48 registers would spill
  static constexpr int warps_target = (P == 1 || P == 3) ? 40 : 32;
  static constexpr int min_blocks = warps_target * 32 / threads > 0 ? warps_target * 32 / threads : 1;
};

// Pairs (a, b), a < b, ordered so that the first n(n-1)/2 use only nodes < n.
__constant__ unsigned char c_pair_a[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
__constant__ unsigned char c_pair_b[10] = {1, 2, 2, 3, 3, 3, 4, 4, 4, 4};

__device__ __forceinline__ int pair_index(int a, int b) {  // a < b
  return b * (b - 1) / 2 + a;
}

// Log-mean factor F with a_log = (aL + aR) / (2 F) and its reciprocal
// (reading R1: Ismail-Roe series for u = f^2 < 1e-4, logarithm otherwise).
// f = (aL - aR)/(aL + aR) is passed in; returns 1/F in *invF and F.  On the
// series branch 1/F is the reciprocal series 1 - u/3 - 4u^2/45 - 44u^3/945
// (from F (1/F) = 1 term by term; the first omitted term is below 1e-17).
// On the logarithm branch log(aL/aR) is taken as lL - lR from per-node
// logarithms when the block has them (have_logs; R1 allows it: the two differ
// by ~1e-14 relative there), else as log(aL/aR); F = log/(2f) and
// 1/F = 2f/log by refined reciprocals (|f| >= 0.01 and |log| >= 0.02 here).
__device__ __forceinline__ double logmean_factor(double aL, double aR, double f, bool have_logs, double lL,
                                                 double lR, double* invF) {
  double u = f * f;
  // u >= 0: the branch test compares bit patterns (integer pipe), equal to u < 1e-4
  if (__double_as_longlong(u) < __double_as_longlong(1e-4)) {
    *invF = fma(u, fma(u, fma(u, -44.0 / 945.0, -4.0 / 45.0), -1.0 / 3.0), 1.0);
    return fma(u, fma(u, fma(u, 1.0 / 7.0, 1.0 / 5.0), 1.0 / 3.0), 1.0);
  }
  const double lz = have_logs ? lL - lR : log(aL / aR);
  *invF = 2.0 * f * rcp(lz);
  return 0.5 * lz * rcp(f);
}

// Whether node value x of an element needs the logarithm branch against the
// element's reference node value r: a pair (a, b) of the element takes the
// logarithm branch only if a/b >= 1.0202 or <= 1/1.0202 (|f| >= 0.01), which
// needs two nodes whose ratio is that large.  For positive doubles the bit
// patterns are monotone and one ulp is a relative step of at most 2^-52, so
// |bits(x) - bits(r)| < 0.0099 2^52 gives x/r within exp(+-0.0099) and any
// pair of such nodes a ratio below exp(0.0198) = 1.0200 < 1.0202 (integer
// pipe only).  Non-positive or NaN values give huge differences: logs are
// taken (and are NaN where the value is, as the pair formula would be).
__device__ __forceinline__ bool far_from_reference(double x, double r) {
  const long long d = __double_as_longlong(x) - __double_as_longlong(r);
  constexpr long long lim = 44585636310967LL;  // 0.0099 * 2^52, rounded down
  return d >= lim || d <= -lim;
}

// Twice the LLF flux, 2 F* = F(U-) + F(U+) - lam (U+ - U-) (the factor 1/2 is
// carried by the volume kernel's end-node coefficient).
__device__ __forceinline__ void llf_flux2_dev(int d, const double* Um, const double* Up, double g, double* F) {
  double im = rcp(Um[0]), ip = rcp(Up[0]);
  double udm = Um[1 + d] * im, udp = Up[1 + d] * ip;
  double pm = (g - 1.0) * (Um[4] - 0.5 * (Um[1] * Um[1] + Um[2] * Um[2] + Um[3] * Um[3]) * im);
  double pp = (g - 1.0) * (Up[4] - 0.5 * (Up[1] * Up[1] + Up[2] * Up[2] + Up[3] * Up[3]) * ip);
  double sm = fabs(udm) + fsqrt(g * pm * im);
  double sp = fabs(udp) + fsqrt(g * pp * ip);
  double lam = fmax(sm, sp);
  double Fm[5], Fp[5];
  Fm[0] = Um[1 + d]; Fp[0] = Up[1 + d];
  Fm[1] = Um[1] * udm + (d == 0 ? pm : 0.0); Fp[1] = Up[1] * udp + (d == 0 ? pp : 0.0);
  Fm[2] = Um[2] * udm + (d == 1 ? pm : 0.0); Fp[2] = Up[2] * udp + (d == 1 ? pp : 0.0);
  Fm[3] = Um[3] * udm; Fp[3] = Up[3] * udp;
  Fm[4] = (Um[4] + pm) * udm; Fp[4] = (Up[4] + pp) * udp;
#pragma unroll
  for (int c = 0; c < 5; ++c) F[c] = fma(-lam, Up[c] - Um[c], Fm[c] + Fp[c]);
}

template <int P>
__global__ void __launch_bounds__(256) k_face(const double* __restrict__ S, double* __restrict__ Fx,
                                              double* __restrict__ Fy, Mesh M) {
  constexpr int n = P + 1, n2 = n * n;
  const size_t N = (size_t)M.K * n2;
  const size_t nf = (size_t)M.K * n;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nf) return;
  int d = t >= nf;
  size_t r = d ? t - nf : t;
  int k = (int)(r / n), j = (int)(r % n);
  int ex = k % M.nx, ey = k / M.nx;
  int km, qm, qp;
  if (d == 0) { km = ey * M.nx + wrap(ex - 1, M.nx); qm = j * n + P; qp = j * n; }
  else { km = wrap(ey - 1, M.ny) * M.nx + ex; qm = P * n + j; qp = j; }
  double Um[5], Up[5], F[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    Um[c] = S[MHD_CHK(c * N + (size_t)km * n2 + qm, 5 * N)];
    Up[c] = S[MHD_CHK(c * N + (size_t)k * n2 + qp, 5 * N)];
  }
  llf_flux2_dev(d, Um, Up, M.g, F);
  double* out = d ? Fy : Fx;
#pragma unroll
  for (int c = 0; c < 5; ++c) out[MHD_CHK(c * nf + r, 5 * nf)] = F[c];
}

// mode 0: write L_E; mode 1: SSP stage combination into C.
// Stage s: s == 0: C = S + tau L; otherwise C = a U0 + b (S + tau L).
template <int P, int MODE, int EBv>
__global__ void __launch_bounds__(HCfg<P, EBv>::threads, HCfg<P, EBv>::min_blocks) k_vol(const double* __restrict__ S, const double* __restrict__ U0,
                                                          const double* __restrict__ Fx, const double* __restrict__ Fy,
                                                          double* __restrict__ out, double* __restrict__ avg_out,
                                                          unsigned* __restrict__ status, const Tab* __restrict__ T,
                                                          Mesh M, const double* __restrict__ dtp, double dtfac,
                                                          double ca, double cb, int first) {
  using C = HCfg<P, EBv>;
  constexpr int n = C::n, n2 = C::n2, EB = C::EB, NP = C::npairs, NPL = C::npl;
  __shared__ double sp[6][EB * n2];           // rho/2, ux/2, uy/2, uz/2, beta, |u|^2/2
  __shared__ double sl[2][EB * n2];           // log(rho/2), log(beta/2), when a pair needs them
  __shared__ double sf[5][EB * NP];           // pair fluxes
  __shared__ double savg[5][EB];
  __shared__ double sDs[2][n2];               // s (-4/h_I) D: the gather rows of both directions, scaled
  __shared__ double sFs[2];                   // s (1/h_I) / w_0: the end-node coefficients of 2 F*, scaled
  const size_t N = (size_t)M.K * n2;
  const int tid = threadIdx.x;
  const int el = tid / n2, q = tid % n2;
  const int k = blockIdx.x * EB + el;
  const bool valid = k < M.K;
  const int kk = valid ? k : M.K - 1;  // clamp loads; results of invalid lanes are discarded
  const size_t gi = (size_t)kk * n2 + q;
  const double g = M.g;

  double Us[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) Us[c] = S[MHD_CHK(c * N + gi, 5 * N)];
  // the gather's coefficients once per block: D and the end-node factors
  // times the metric and, in the stage combination, times tau (first stage)
  // or b tau, so that the gather yields the stage increment directly
  {
    const double sc = MODE == 0 ? 1.0 : (first ? dtp[0] * dtfac : cb * (dtp[0] * dtfac));
    constexpr double w0i = 0.5 * P * (P + 1);  // 1 / w_0 of GLL(p): w_0 = 2 / (p (p + 1))
    const double sx = -4.0 * M.ihx * sc, sy = -4.0 * M.ihy * sc;
    for (int t = tid; t < 2 * n2 + 2; t += EB * n2) {
      if (t < 2 * n2) sDs[t / n2][t % n2] = T->D[(t % n2) / n][t % n] * (t < n2 ? sx : sy);
      else sFs[t - 2 * n2] = (t == 2 * n2 ? M.ihx : M.ihy) * w0i * sc;  // (2/h) / w_0 times F* = (1/h) / w_0 times 2 F*
    }
  }
  {
    // halves: the pair means {{.}} become plain sums.  Scaling by powers of 2
    // is exact, so v = u/2 = m (1/(2 rho)), q = |v|^2 = |u|^2/4 and
    // -2 rho q = -rho |u|^2 / 2 are the same doubles as the unscaled forms
    const double hir = 0.5 * rcp(Us[0]);
    const double vx = Us[1] * hir, vy = Us[2] * hir, vz = Us[3] * hir;
    const double q4 = fma(vx, vx, fma(vy, vy, vz * vz));
    const double pr = (g - 1.0) * fma(-2.0 * Us[0], q4, Us[4]);
    const double hr = 0.5 * Us[0];
    sp[0][tid] = hr;
    sp[1][tid] = vx; sp[2][tid] = vy; sp[3][tid] = vz;
    sp[4][tid] = hr * rcp(pr);
    sp[5][tid] = 2.0 * q4;
  }
  __syncthreads();
  // per-node logarithms for the whole block, only if some element of it has a
  // node far enough from its first node for a pair to take the log branch
  // (one block vote; the block's threads take the same branch)
  const bool far = far_from_reference(sp[0][tid], sp[0][el * n2]) || far_from_reference(sp[4][tid], sp[4][el * n2]);
  const bool have_logs = __syncthreads_or(far) != 0;
  if (have_logs) {
    sl[0][tid] = log(sp[0][tid]);
    sl[1][tid] = log(sp[4][tid]);
    __syncthreads();
  }

  // ---- pair fluxes ------------------------------------------------------------
  const double ig1 = M.ig1;
#pragma unroll
  for (int s = 0; s < P; ++s) {
    const int pidx = q + s * n2;
    const int d = pidx >= NP / 2;
    const int r = pidx - d * (NP / 2);
    const int line = r / NPL, w = r % NPL;
    const int a = c_pair_a[w], b = c_pair_b[w];
    const int qa = (int)MHD_CHK(el * n2 + (d == 0 ? line * n + a : a * n + line), EB * n2);
    const int qb = (int)MHD_CHK(el * n2 + (d == 0 ? line * n + b : b * n + line), EB * n2);
    double rL = sp[0][qa], rR = sp[0][qb];              // rho/2 of both nodes
    double bL = sp[4][qa], bR = sp[4][qb];
    double hr = rL + rR, sb = bL + bR;                  // {{rho}}, 2 {{beta}}
    double isr = rcp(hr), isb = rcp(sb);
    double fr = (rL - rR) * isr, fb = (bL - bR) * isb;
    double iFr, iFb;
    double Fr = have_logs ? logmean_factor(rL, rR, fr, true, sl[0][qa], sl[0][qb], &iFr)
                          : logmean_factor(rL, rR, fr, false, 0.0, 0.0, &iFr);
    double Fb = have_logs ? logmean_factor(bL, bR, fb, true, sl[1][qa], sl[1][qb], &iFb)
                          : logmean_factor(bL, bR, fb, false, 0.0, 0.0, &iFb);
    double rlog = hr * iFr;                             // rho^log
    double ua0 = sp[1][qa] + sp[1][qb];
    double ua1 = sp[2][qa] + sp[2][qb];
    double ua2 = sp[3][qa] + sp[3][qb];
    double u2a = sp[5][qa] + sp[5][qb];                 // {{|u|^2}}
    double au2 = fma(ua0, ua0, fma(ua1, ua1, ua2 * ua2));  // |{{u}}|^2
    double phat = hr * isb;                             // {{rho}} / (2 {{beta}})
    // h = 1/(2(g-1) beta^log) - {{|u|^2}}/2 + |{{u}}|^2 + phat/rho^log
    //   = Fb/((g-1) sb) ... with beta^log = sb/(2 Fb) and rho^log = sr/(2 Fr)
    double hhat = fma(Fb * ig1 + Fr, isb, fma(-0.5, u2a, au2));
    double ud = d == 0 ? ua0 : ua1;
    double f0 = rlog * ud;
    const int o = (int)MHD_CHK(el * NP + pidx, EB * NP);
    sf[0][o] = f0;
    sf[1][o] = fma(f0, ua0, d == 0 ? phat : 0.0);
    sf[2][o] = fma(f0, ua1, d == 1 ? phat : 0.0);
    sf[3][o] = f0 * ua2;
    sf[4][o] = f0 * hhat;
  }
  __syncthreads();

  // ---- gather: L = -(2/hx)[2 sum D F + end terms] - (2/hy)[...] -----------------
  // (times the block's scale s: 1 for the residual, tau or b tau in a stage)
  const int i = q % n, j = q / n;
  // the p off-diagonal terms of rows i and j of D, visited as r = i + o (mod n),
  // o = 1..p: no lane-dependent skip of the diagonal, so no predicated-off FMA
  double Dx[P], Dy[P];
  int px[P], py[P];
#pragma unroll
  for (int o = 1; o < n; ++o) {
    const int rx = i + o < n ? i + o : i + o - n, ry = j + o < n ? j + o : j + o - n;
    Dx[o - 1] = sDs[0][i * n + rx];
    Dy[o - 1] = sDs[1][j * n + ry];
    px[o - 1] = (int)MHD_CHK(el * NP + j * NPL + pair_index(min(i, rx), max(i, rx)), EB * NP);
    py[o - 1] = (int)MHD_CHK(el * NP + NP / 2 + i * NPL + pair_index(min(j, ry), max(j, ry)), EB * NP);
  }
  const int ex = kk % M.nx, ey = kk / M.nx;
  const size_t nf = (size_t)M.K * n;
  // face terms as one FMA per direction in every lane: the coefficient of 2 F*
  // is +-1/(h w_0) on the end nodes and 0 inside (0 * F* adds an exact zero),
  // so no lane-divergent block is issued
  const double cfx = i == 0 ? sFs[0] : (i == P ? -sFs[0] : 0.0);
  const double cfy = j == 0 ? sFs[1] : (j == P ? -sFs[1] : 0.0);
  const size_t ifx = (i == P ? (size_t)(ey * M.nx + wrap(ex + 1, M.nx)) : (size_t)kk) * n + j;
  const size_t ify = (j == P ? (size_t)(wrap(ey + 1, M.ny) * M.nx + ex) : (size_t)kk) * n + i;
  double L[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    // one chain over both directions (the rows carry the metric factors)
    double v = 0.0;
#pragma unroll
    for (int o = 0; o < P; ++o) v = fma(Dx[o], sf[c][px[o]], v);
#pragma unroll
    for (int o = 0; o < P; ++o) v = fma(Dy[o], sf[c][py[o]], v);
    // end nodes: -(2/hx)[-F*_left/w_0] and -(2/hx)[+F*_right/w_p] (w_p = w_0)
    v = fma(cfx, Fx[MHD_CHK(c * nf + ifx, 5 * nf)], v);
    v = fma(cfy, Fy[MHD_CHK(c * nf + ify, 5 * nf)], v);
    L[c] = v;
  }

  if constexpr (MODE == 0) {
    if (valid) {
#pragma unroll
      for (int c = 0; c < 5; ++c) out[MHD_CHK(c * N + gi, 5 * N)] = L[c];
    }
  } else {
    // L is tau L (first stage) or b tau L: C = S + tau L, or a U0 + b S + b tau L
    double Cv[5];
#pragma unroll
    for (int c = 0; c < 5; ++c)
      Cv[c] = first ? Us[c] + L[c] : fma(ca, U0[MHD_CHK(c * N + gi, 5 * N)], fma(cb, Us[c], L[c]));
    if (valid) {
#pragma unroll
      for (int c = 0; c < 5; ++c) out[MHD_CHK(c * N + gi, 5 * N)] = Cv[c];
    }
    // no status word: the caller's limiter tests the same averages itself (the
    // OE before it keeps them), so the reduction below is skipped (block-uniform)
    if (status == nullptr && avg_out == nullptr) return;
    // ---- raw element averages and the admissibility check --------------------------
    double a0, a1, a2, a3, a4;
    if constexpr (n2 == 4 || n2 == 16) {
      // an element is an aligned power-of-two lane segment: xor-shuffle sums
      const double wq = 0.25 * T->wp[i] * T->wp[j];
      double w[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) w[c] = wq * Cv[c];
#pragma unroll
      for (int o = n2 / 2; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 5; ++c) w[c] += __shfl_xor_sync(0xffffffffu, w[c], o);
      a0 = w[0]; a1 = w[1]; a2 = w[2]; a3 = w[3]; a4 = w[4];
    } else {
      __syncthreads();  // sf is reused for the stage values
#pragma unroll
      for (int c = 0; c < 5; ++c) sf[c][el * n2 + q] = Cv[c];
      __syncthreads();
      // component c is reduced by node thread c mod n2
      for (int c = q; c < 5; c += n2) {
        double s = 0.0;
#pragma unroll
        for (int t2 = 0; t2 < n2; ++t2) s = fma(0.25 * T->wp[t2 % n] * T->wp[t2 / n], sf[c][el * n2 + t2], s);
        savg[c][el] = s;
      }
      __syncthreads();
      a0 = savg[0][el]; a1 = savg[1][el]; a2 = savg[2][el]; a3 = savg[3][el]; a4 = savg[4][el];
    }
    if (q == 0 && valid) {
      if (avg_out) {
        avg_out[0 * (size_t)M.K + k] = a0; avg_out[1 * (size_t)M.K + k] = a1; avg_out[2 * (size_t)M.K + k] = a2;
        avg_out[3 * (size_t)M.K + k] = a3; avg_out[4 * (size_t)M.K + k] = a4;
      }
      // rho > 0 and p > 0  <=>  rho > 0 and rho E - |m|^2/2 > 0
      double pe = fma(a0, a4, -0.5 * fma(a1, a1, fma(a2, a2, a3 * a3)));
      bool fin = isfinite(a0) && isfinite(a1) && isfinite(a2) && isfinite(a3) && isfinite(a4);
      if (status) {
        if (!fin) atomicOr(status, ST_NONFINITE | ST_INADMISSIBLE);
        else if (!(a0 > 0.0) || !(pe > 0.0)) atomicOr(status, ST_INADMISSIBLE);
      }
    }
  }
}

// ---- launchers ------------------------------------------------------------------
template <int P>
void launch_face(const double* S, double* Fx, double* Fy, const Mesh& M, cudaStream_t st) {
  size_t total = 2 * (size_t)M.K * (P + 1);
  int th = 256;
  k_face<P><<<(unsigned)((total + th - 1) / th), th, 0, st>>>(S, Fx, Fy, M);
}

template <int P, int EBv>
void launch_vol_eb(int mode, const double* S, const double* U0, const double* Fx, const double* Fy, double* out,
                   double* avg, unsigned* status, const Tab* T, const Mesh& M, const double* dtp, double dtfac,
                   double ca, double cb, int first, cudaStream_t st) {
  using C = HCfg<P, EBv>;
  unsigned blocks = (unsigned)((M.K + C::EB - 1) / C::EB);
  if (mode == 0)
    k_vol<P, 0, EBv><<<blocks, C::threads, 0, st>>>(S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb,
                                                   first);
  else
    k_vol<P, 1, EBv><<<blocks, C::threads, 0, st>>>(S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb,
                                                   first);
}

template <int P>
void launch_vol(int mode, const double* S, const double* U0, const double* Fx, const double* Fy, double* out,
                double* avg, unsigned* status, const Tab* T, const Mesh& M, const double* dtp, double dtfac,
                double ca, double cb, int first, cudaStream_t st) {
  switch (M.tile_vol) {
    case 1: launch_vol_eb<P, vol_tile_eb(P, 1)>(mode, S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb, first, st); break;
    case 2: launch_vol_eb<P, vol_tile_eb(P, 2)>(mode, S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb, first, st); break;
    default: launch_vol_eb<P, vol_tile_eb(P, 0)>(mode, S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb, first, st); break;
  }
}

void hydro_face(int p, const double* S, double* Fx, double* Fy, const Mesh& M, cudaStream_t st) {
  switch (p) {
    case 1: launch_face<1>(S, Fx, Fy, M, st); break;
    case 2: launch_face<2>(S, Fx, Fy, M, st); break;
    case 3: launch_face<3>(S, Fx, Fy, M, st); break;
    case 4: launch_face<4>(S, Fx, Fy, M, st); break;
  }
}

void hydro_vol(int p, int mode, const double* S, const double* U0, const double* Fx, const double* Fy, double* out,
               double* avg, unsigned* status, const Tab* T, const Mesh& M, const double* dtp, double dtfac,
               double ca, double cb, int first, cudaStream_t st) {
  switch (p) {
    case 1: launch_vol<1>(mode, S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb, first, st); break;
    case 2: launch_vol<2>(mode, S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb, first, st); break;
    case 3: launch_vol<3>(mode, S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb, first, st); break;
    case 4: launch_vol<4>(mode, S, U0, Fx, Fy, out, avg, status, T, M, dtp, dtfac, ca, cb, first, st); break;
  }
}

MHD_OOB_READER(oob_hydro)

}  // namespace mhd
