// Stage stabilisation kernels.
//
//  * Hydro stage map P = P_PP o P_OE (§3.2.2): direction-resolved jump sensor
//    with cross-line scaling (eqs. euler-oe-jump, euler-oe-amplitude,
//    euler-oe-shared-amplitude, euler-oe-sigma), damping of the discrete
//    Legendre shells (eqs. euler-oe-rate, euler-oe-factor, euler-oe-map) and
//    the Zhang-Shu scaling limiter (eqs. euler-pp-*).
//  * Artificial-resistivity coefficient (eqs. magnetic-ar-sensor,
//    magnetic-ar-coefficient), once per magnetic substep.
//  * Velocity OE (eqs. magnetic-oe-sensor, magnetic-oe-rate,
//    magnetic-oe-factor, magnetic-oe-map): rho-weighted nested projections
//    through Psi = Phi L^{-T} (G = Phi^T W Phi = L L^T), built once per substep.
//
// The sensor statistics are shared by both OE procedures: k_stats writes per
// element and component the average, nodal max/min and the jump measures of
// its -x and -y faces; k_lines reduces rows and columns in a fixed order;
// k_global reduces the rows and tabulates the reciprocal shared amplitude of
// every row and column and the order factors of the sensor.  Readings R6-R9 of
// the design notes apply.
#include <cfloat>
#include <cmath>
#include <vector>

#include "mhd_internal.cuh"

namespace mhd {

// ---- work-buffer layout ---------------------------------------------------------
struct StatsView {
  double* avg;   // [nc][K]
  double* emax;  // [nc][K]
  double* emin;  // [nc][K]
  double* jx;    // [nc][n][K] jump measure of the -x face of element K
  double* jy;    // [nc][n][K] jump measure of the -y face
  double* line;  // [2][L][nc][3]: (sum of averages, max, min) per row (0) / column (1), L = max(nx, ny)
  double* glob;  // [nc][4]: mean, amplitude Delta_Omega, L-inf norm, roundoff-constant flag
  double* ar;    // [K][8] A.R. per-element partials
  double* arg;   // [8] A.R. global values
  double* part;  // [ceil(K/256)][9] A.R. chunk partials
  double* lineD; // [2][L] 1 / Delta_{I,line} (eq. euler-oe-shared-amplitude), from k_global
  double* rfac;  // [2][8] (2r + 1) h_I^r / (2 r!) of eq. euler-oe-sigma, from k_global
  // per-mesh coefficients of the face jumps (set at context creation, stab_init_mesh):
  double* jcoef; // [2 (I)][2 (side: 0 this element's lower face, 1 the neighbour's upper face)][p][n][n]:
                 //   sqrt(w_t / 2) (2/h_I)^r times row 0 (side 0) or minus row p (side 1) of D^r, r = 1..p
  double* sqw;   // [n] sqrt(w_t / 2)
};

static StatsView stats_view(double* work, int p, const Mesh& M) {
  const size_t K = M.K, n = p + 1, L = M.nx > M.ny ? M.nx : M.ny;
  const size_t NC = 5;
  StatsView v;
  v.avg = work;
  v.emax = v.avg + NC * K;
  v.emin = v.emax + NC * K;
  v.jx = v.emin + NC * K;
  v.jy = v.jx + NC * n * K;
  v.line = v.jy + NC * n * K;
  v.glob = v.line + 2 * L * NC * 3;
  v.ar = v.glob + NC * 4;
  v.arg = v.ar + 8 * K;
  v.part = v.arg + 8;
  v.lineD = v.part + 9 * (K / 256 + 1);
  v.rfac = v.lineD + 2 * L;
  v.jcoef = v.rfac + 16;
  v.sqw = v.jcoef + 4 * p * n * n;
  return v;
}

size_t stab_work_doubles(int p, int k, const Mesh& M) {
  (void)k;
  const size_t K = M.K, n = p + 1, L = M.nx > M.ny ? M.nx : M.ny;
  return 3 * 5 * K + 2 * 5 * n * K + 2 * L * 5 * 3 + 5 * 4 + 8 * K + 8 + 9 * (K / 256 + 1) + 2 * L + 16 +
         4 * p * n * n + n + 64;
}

// The face-jump coefficients of a mesh into the work buffer (once per context).
cudaError_t stab_init_mesh(int p, const Tab& hT, const Mesh& M, double* work) {
  const StatsView V = stats_view(work, p, M);
  const int n = p + 1;
  std::vector<double> c(4 * p * n * n + n);
  double* jc = c.data();
  double* sq = jc + 4 * p * n * n;
  for (int t = 0; t < n; ++t) sq[t] = sqrt(hT.hwp[t]);
  for (int I = 0; I < 2; ++I) {
    const double s2h = 2.0 * (I == 0 ? M.ihx : M.ihy);
    for (int r = 1; r <= p; ++r) {
      double scale = 1.0;
      for (int i = 0; i < r; ++i) scale *= s2h;
      for (int t = 0; t < n; ++t)
        for (int q = 0; q < n; ++q) {
          jc[(((I * 2 + 0) * p + (r - 1)) * n + t) * n + q] = sq[t] * scale * hT.Dr0[r][q];
          jc[(((I * 2 + 1) * p + (r - 1)) * n + t) * n + q] = -(sq[t] * scale * hT.Drp[r][q]);
        }
    }
  }
  return cudaMemcpy(V.jcoef, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice);
}

size_t stab_chol_doubles(int p, const Mesh& M) {
  const size_t n2 = (size_t)(p + 1) * (p + 1);
  return (size_t)M.K * n2 * n2;
}

// ---- k_stats: per element and component --------------------------------------------
// One thread per (component, item, element), element fastest: item 0 the
// weighted average and the nodal max and min; items 1 and 2 the jump measures
// J_r, r = 0..p, of the lower face normal to x and to y (eq. euler-oe-jump),
// from one load of the two elements' nodes.  The face quadrature weight and
// (2/h)^r are folded into the derivative rows (V.jcoef), so a face node's
// weighted jump of order r is one chain of 2 (p+1) FMAs and its square one more.
template <int P, int I>
__device__ __forceinline__ void face_jumps(const double* __restrict__ f, int k, int kA, const StatsView& V,
                                           double* __restrict__ out, size_t K, int c) {
  constexpr int n = P + 1, n2 = n * n;
  const double* cB = V.jcoef + (size_t)(I * 2 + 0) * P * n * n;
  const double* cA = V.jcoef + (size_t)(I * 2 + 1) * P * n * n;
  double acc[n];
#pragma unroll
  for (int r = 0; r < n; ++r) acc[r] = 0.0;
  // face node t: the normal line t of both elements (x-direction rows, y-direction
  // columns), then the weighted jumps of every order, accumulated in t order
#pragma unroll
  for (int t = 0; t < n; ++t) {
    double a[n], b[n];
#pragma unroll
    for (int s = 0; s < n; ++s) {
      const int q = I == 0 ? t * n + s : s * n + t;
      a[s] = f[MHD_CHK((size_t)kA * n2 + q, K * n2)];
      b[s] = f[MHD_CHK((size_t)k * n2 + q, K * n2)];
    }
    {  // r = 0: the traces themselves
      const double jw = V.sqw[t] * (b[0] - a[P]);
      acc[0] = fma(jw, jw, acc[0]);
    }
#pragma unroll
    for (int r = 1; r <= P; ++r) {
      double jw = 0.0;
#pragma unroll
      for (int s = 0; s < n; ++s) jw = fma(cB[((r - 1) * n + t) * n + s], b[s], jw);
#pragma unroll
      for (int s = 0; s < n; ++s) jw = fma(cA[((r - 1) * n + t) * n + s], a[s], jw);
      acc[r] = fma(jw, jw, acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < n; ++r) out[MHD_CHK(((size_t)c * n + r) * K + k, 5 * n * K)] = fsqrt(acc[r]);
}

template <int P>
__global__ void __launch_bounds__(256) k_stats(const double* __restrict__ F, size_t stride, int nc, StatsView V,
                                               const Tab* __restrict__ T, Mesh M) {
  constexpr int n = P + 1, n2 = n * n;
  const size_t K = M.K;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nc * 3 * K) return;
  const int k = (int)(t % K);
  const int it = (int)(t / K);
  const int c = it / 3, w = it % 3;
  const double* f = F + c * stride;
  const int ex = k % M.nx, ey = k / M.nx;
  if (w == 0) {  // weighted average; nodal max and min on integer keys
    double s = 0.0;
    long long mx = dkey(-DBL_MAX), mn = dkey(DBL_MAX);
#pragma unroll
    for (int q = 0; q < n2; ++q) {
      double v = f[(size_t)k * n2 + q];
      s = fma(T->Wq[q], v, s);
      const long long kv = dkey(v);
      mx = kv > mx ? kv : mx;
      mn = kv < mn ? kv : mn;
    }
    V.avg[c * K + k] = s;
    V.emax[c * K + k] = dkey_inv(mx);
    V.emin[c * K + k] = dkey_inv(mn);
    return;
  }
  if (w == 1) face_jumps<P, 0>(f, k, ey * M.nx + wrap(ex - 1, M.nx), V, V.jx, K, c);
  else face_jumps<P, 1>(f, k, wrap(ey - 1, M.ny) * M.nx + ex, V, V.jy, K, c);
}

// ---- k_lines: row (blockIdx.y = 0) and column (1) reductions -----------------------
// Fixed-order tree: thread t accumulates a strided subset, then a pairwise tree.
__global__ void k_lines(int nc, StatsView V, Mesh M) {
  const int dir = blockIdx.y, L = blockIdx.x;
  const int nlines = dir == 0 ? M.ny : M.nx, len = dir == 0 ? M.nx : M.ny;
  if (L >= nlines) return;
  const size_t K = M.K;
  const int Lmax = M.nx > M.ny ? M.nx : M.ny;
  __shared__ double s_sum[256], s_max[256], s_min[256];
  for (int c = 0; c < nc; ++c) {
    double s = 0.0, mx = -DBL_MAX, mn = DBL_MAX;
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
      int k = (int)MHD_CHK(dir == 0 ? L * M.nx + t : t * M.nx + L, K);
      s += V.avg[c * K + k];
      mx = fmax(mx, V.emax[c * K + k]);
      mn = fmin(mn, V.emin[c * K + k]);
    }
    s_sum[threadIdx.x] = s; s_max[threadIdx.x] = mx; s_min[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
        s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
        s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double* o = V.line + (((size_t)dir * Lmax + L) * nc + c) * 3;
      o[0] = s_sum[0]; o[1] = s_max[0]; o[2] = s_min[0];
    }
    __syncthreads();
  }
}

// ---- k_global: from the row reductions --------------------------------------------
__global__ void k_global(int nc, int n, StatsView V, Mesh M) {
  __shared__ double s_sum[256], s_max[256], s_min[256];
  const int Lmax = M.nx > M.ny ? M.nx : M.ny;
  for (int c = 0; c < nc; ++c) {
    double s = 0.0, mx = -DBL_MAX, mn = DBL_MAX;
    for (int L = threadIdx.x; L < M.ny; L += blockDim.x) {
      const double* o = V.line + ((size_t)L * nc + c) * 3;
      s += o[0]; mx = fmax(mx, o[1]); mn = fmin(mn, o[2]);
    }
    s_sum[threadIdx.x] = s; s_max[threadIdx.x] = mx; s_min[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
        s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
        s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double mean = s_sum[0] / M.K;
      double amp = fmax(s_max[0] - mean, mean - s_min[0]);
      double linf = fmax(fabs(s_max[0]), fabs(s_min[0]));
      double* g = V.glob + c * 4;
      g[0] = mean; g[1] = amp; g[2] = linf;
      g[3] = amp <= 1024.0 * DBL_EPSILON * fmax(linf, 1e-300) ? 1.0 : 0.0;  // reading R8
    }
    __syncthreads();
  }
  // 1 / Delta_{I,L} of every row (I = 0) and column (I = 1), with the global
  // amplitude floor, and the order factors of the sensor
  for (int t = threadIdx.x; t < 2 * Lmax; t += blockDim.x) {
    const int I = t / Lmax, L = t % Lmax;
    const int nl = I == 0 ? M.ny : M.nx, len = I == 0 ? M.nx : M.ny;
    if (L >= nl) continue;
    const double ilen = 1.0 / len;
    double D = 0.0;
    for (int c = 0; c < nc; ++c) {
      const double* o = V.line + (((size_t)I * Lmax + L) * nc + c) * 3;
      const double mean = o[0] * ilen;
      const double amp = fmax(o[1] - mean, mean - o[2]);
      D = fmax(D, fmax(amp, 1e-6 * V.glob[c * 4 + 1]));
    }
    // D = 0 only when every component is constant to roundoff (reading R8);
    // then no component enters sigma, which is 0: keep 0 * (1/D) finite
    V.lineD[t] = D > 0.0 ? 1.0 / D : 0.0;
  }
  if (threadIdx.x < 2 * n) {
    const int I = threadIdx.x / n, r = threadIdx.x % n;
    const double h = I == 0 ? M.hx : M.hy;
    double hr = 1.0, fact = 1.0;
    for (int i = 0; i < r; ++i) { hr *= h; fact *= (i + 1); }
    V.rfac[I * 8 + r] = (2.0 * r + 1.0) * hr / (2.0 * fact);
  }
}

// sigma_{r,I,K} (eq. euler-oe-sigma / magnetic-oe-sensor): max over the
// components not constant to roundoff (reading R8; the flag is tested on its
// bit pattern) of the order factor times the face jump measures of the two
// faces, over the shared amplitude of the element's line.
__device__ __forceinline__ double sigma_rI(const StatsView& V, int nc, int n, int I, int r, int k, int kB,
                                           double iDelta, size_t K) {
  const double* J = I == 0 ? V.jx : V.jy;
  const double fac = V.rfac[I * 8 + r];
  double s = 0.0;
  for (int c = 0; c < nc; ++c) {
    if (__double_as_longlong(V.glob[c * 4 + 3]) != 0) continue;
    const double Jr = J[MHD_CHK(((size_t)c * n + r) * K + k, 5 * n * K)] + J[MHD_CHK(((size_t)c * n + r) * K + kB, 5 * n * K)];
    s = fmax(s, Jr);
  }
  return fac * s * iDelta;
}

// ---- k_oe_pp: hydro OE map then the positivity limiter ----------------------------
// Each element owns a segment of SW lanes (SW = smallest power of two >= (p+1)^2,
// a divisor of 32), so per-element minima, maxima and sums are shuffle trees and
// every lane of the segment carries its node's share of the limiter; the
// scalar per-element quantities are evaluated by all lanes of the segment.
template <int P>
struct OCfg {
  static constexpr int n = P + 1, n2 = n * n;
  static constexpr int SW = n2 <= 4 ? 4 : (n2 <= 16 ? 16 : 32);
  static constexpr int EB = 128 / SW;
  static constexpr int threads = EB * SW;
};

// Segment minimum / maximum on order-preserving integer keys (integer pipe).
template <int SW>
__device__ __forceinline__ double seg_min(double v) {
  long long kv = dkey(v);
#pragma unroll
  for (int o = SW / 2; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, kv, o);
    kv = w < kv ? w : kv;
  }
  return dkey_inv(kv);
}
template <int SW>
__device__ __forceinline__ double seg_max(double v) {
  long long kv = dkey(v);
#pragma unroll
  for (int o = SW / 2; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, kv, o);
    kv = w > kv ? w : kv;
  }
  return dkey_inv(kv);
}
template <int SW>
__device__ __forceinline__ double seg_sum(double v) {
#pragma unroll
  for (int o = SW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-element OE damping factors D_l (eq. euler-oe-factor / magnetic-oe-factor):
// lanes q < 2n evaluate sigma_{r,I} (I = q / n, r = q % n); lanes q < n sum
// Theta_l and take the exponential.  lam[I] must be valid in every lane.
template <int P>
__device__ __forceinline__ void oe_factors(const StatsView& V, int nc, int q, int el, int kk, int ex, int ey,
                                           const double lam[2], double s_tau, const Mesh& M,
                                           double (*ssig)[2 * (P + 1)], double (*sD)[P + 1]) {
  constexpr int n = P + 1;
  if (q < 2 * n) {
    const int I = q / n, r = q % n;
    const int Lmax = M.nx > M.ny ? M.nx : M.ny;
    const double iDelta = V.lineD[I * Lmax + (I == 0 ? ey : ex)];
    const int kB = I == 0 ? ey * M.nx + wrap(ex + 1, M.nx) : wrap(ey + 1, M.ny) * M.nx + ex;
    ssig[el][q] = sigma_rI(V, nc, n, I, r, kk, kB, iDelta, M.K);
  }
  __syncthreads();
  if (q < n) {
    double Theta = 0.0;
    for (int I = 0; I < 2; ++I) {
      double ss = 0.0;
      for (int r = 0; r <= q; ++r) ss += ssig[el][I * n + r];
      Theta = fma(lam[I], ss, Theta);
    }
    sD[el][q] = q == 0 ? 1.0 : exp(-s_tau * Theta);
  }
  __syncthreads();
}

// ---- k_oe_pp: hydro OE map then the positivity limiter ----------------------------
// One thread per node (EB elements x (p+1)^2 threads, no padding).  The node
// work (the sum-factorised modal transform there and back, the nodal parts of
// the limiter) runs in registers; everything that is one value per element or
// per (element, direction, order) - the rate lambda, the sensor sigma, the
// factors D_l, the averages, the limiter's scalars and decisions - runs once
// per element in flat item loops over the block, so that no FP64 instruction
// is spent repeating an element's scalar in every node lane.
template <int P>
struct PCfg {
  static constexpr int n = P + 1, n2 = n * n;
  static constexpr int EB = P == 1 ? 64 : P == 2 ? 28 : P == 3 ? 16 : 10;  // ~256 threads
  static constexpr int threads = EB * n2;
};

// Per-element scalars of the limiter in shared memory.
enum { PE_RBAR = 0, PE_PBAR, PE_SA, PE_THR, PE_EPSP, PE_THP, PE_MODE, PE_TRHO, PE_TALL, PE_N };

// frz (may be null): per element the frozen coefficients of the map, [K][p+3]:
// D_0..D_p of the OE and the limiter factors t_rho (density) and t (others),
// U'' = t U* + (1 - t) avg(U*), for the adjoint.
template <int P>
__global__ void __launch_bounds__(PCfg<P>::threads) k_oe_pp(double* __restrict__ S, StatsView V,
                                                            const Tab* __restrict__ T, Mesh M, Stab prm,
                                                            const double* __restrict__ dtp, double dtfac,
                                                            unsigned* __restrict__ status,
                                                            double* __restrict__ frz) {
  using C = PCfg<P>;
  constexpr int n = C::n, n2 = C::n2, EB = C::EB, TH = C::threads;
  __shared__ double su[5][EB * n2];
  __shared__ double st[5][EB * n2];
  // x-filter rows K_b[i][.] of node (i, b): row stride n + 1 and element stride
  // n2 (n + 1) + 1 (odd), so neither the per-element writes nor the row reads collide in banks
  constexpr int KS = n2 * (n + 1) + 1;
  __shared__ double sK[EB * KS];
  __shared__ double ssig[EB][2 * n];
  __shared__ double sD[EB][n];
  __shared__ double slam[EB][2];
  __shared__ double sa[5][EB];
  __shared__ double se[PE_N][EB];
  const size_t N = (size_t)M.K * n2, K = M.K;
  const int tid = threadIdx.x, el = tid / n2, q = tid % n2;
  const int k0 = blockIdx.x * EB;
  const int k = k0 + el;
  const bool valid = k < M.K;
  const int kk = valid ? k : M.K - 1;
  const int i = q % n, j = q / n;
  const double g = M.g;
  double u[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) u[c] = S[MHD_CHK(c * N + (size_t)kk * n2 + q, 5 * N)];

  if (prm.oe_hydro) {
#pragma unroll
    for (int c = 0; c < 5; ++c) su[c][tid] = u[c];
    // rate lambda_{E,I} (eq. euler-oe-rate) from the element average, once per element
    for (int e = tid; e < EB; e += TH) {
      const int ke = min(k0 + e, M.K - 1);
      const double a0 = V.avg[MHD_CHK(ke, K)], a1 = V.avg[K + ke], a2 = V.avg[2 * K + ke], a3 = V.avg[3 * K + ke],
                   a4 = V.avg[4 * K + ke];
      const double ir = rcp(a0);
      const double pb = (g - 1.0) * fma(-0.5 * ir, fma(a1, a1, fma(a2, a2, a3 * a3)), a4);
      const double cb = fsqrt(g * pb * ir);
      slam[e][0] = (2.0 * P + 1.0) * (fabs(a1 * ir) + cb) * M.ihx;
      slam[e][1] = (2.0 * P + 1.0) * (fabs(a2 * ir) + cb) * M.ihy;
    }
    // sigma_{r,I} (eq. euler-oe-sigma), once per (element, direction, order)
    const int Lmax = M.nx > M.ny ? M.nx : M.ny;
    for (int it = tid; it < EB * 2 * n; it += TH) {
      const int e = it / (2 * n), w = it % (2 * n), I = w / n, r = w % n;
      const int ke = min(k0 + e, M.K - 1), ex = ke % M.nx, ey = ke / M.nx;
      const double iDelta = V.lineD[I * Lmax + (I == 0 ? ey : ex)];
      const int kB = I == 0 ? ey * M.nx + wrap(ex + 1, M.nx) : wrap(ey + 1, M.ny) * M.nx + ex;
      ssig[e][w] = sigma_rI(V, 5, n, I, r, ke, kB, iDelta, K);
    }
    __syncthreads();
    // D_l = exp(-s_H tau Theta_l) (eq. euler-oe-factor), once per (element, shell)
    const double s_tau = prm.s_H * dtp[0] * dtfac;
    for (int it = tid; it < EB * n; it += TH) {
      const int e = it / n, l = it % n;
      double Theta = 0.0;
      for (int I = 0; I < 2; ++I) {
        double ss = 0.0;
        for (int r = 0; r <= l; ++r) ss += ssig[e][I * n + r];
        Theta = fma(slam[e][I], ss, Theta);
      }
      sD[e][l] = l == 0 ? 1.0 : exp(-s_tau * Theta);
    }
    __syncthreads();
    {  // T[b][i] = sum_j w_j P_b(x_j) U[j][i]   (b = j of this thread)
      double wl[n];
#pragma unroll
      for (int jj = 0; jj < n; ++jj) wl[jj] = T->WLeg[jj][j];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double v = 0.0;
#pragma unroll
        for (int jj = 0; jj < n; ++jj) v = fma(wl[jj], su[c][el * n2 + jj * n + i], v);
        st[c][tid] = v;
      }
    }
    // the x-direction filter of every y-mode b, once per element and shared by
    // the five fields: K_b[i][i'] = sum_a D_max(a,b) N_a N_b P_a(x_i) w_i' P_a(x_i')
    // (forward x-transform, damping and backward x-transform in one n x n matrix);
    // items (b, i, i') element-fastest, so a warp's items share b and its cost
    for (int it = tid; it < EB * n * n2; it += TH) {
      const int e = it % EB, w = it / EB, b = w / n2, r = w % n2, ii = r / n, i2 = r % n;
      double v = sD[e][b] * T->OES[b][ii][i2];
      for (int a = b + 1; a < n; ++a) v = fma(sD[e][a], T->OEQ[b][a][ii][i2], v);
      sK[e * KS + (b * n + ii) * (n + 1) + i2] = v;
    }
    __syncthreads();
    // V[b][i] = sum_i' K_b[i][i'] T[b][i']   (b = j of this thread)
    {
      double kr[n];
#pragma unroll
      for (int i2 = 0; i2 < n; ++i2) kr[i2] = sK[el * KS + (j * n + i) * (n + 1) + i2];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double v = 0.0;
#pragma unroll
        for (int i2 = 0; i2 < n; ++i2) v = fma(kr[i2], st[c][el * n2 + j * n + i2], v);
        su[c][tid] = v;
      }
    }
    __syncthreads();
    // U[j][i] = sum_b P_b(x_j) V[b][i]
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < n; ++b) v = fma(T->Leg[j][b], su[c][el * n2 + b * n + i], v);
      u[c] = v;
    }
    __syncthreads();  // su and st are reused below
  }

  double t_rho = 1.0, t_all = 1.0;  // frozen limiter factors (adjoint)
  if (prm.pp) {
    const double eps = DBL_EPSILON, eps_rho = 64.0 * eps;
#pragma unroll
    for (int c = 0; c < 5; ++c) su[c][tid] = u[c];
    __syncthreads();
    // element averages of U* (eq. euler-pp-average), once per (element, component)
    for (int it = tid; it < EB * 5; it += TH) {
      const int e = it / 5, c = it % 5;
      double s = 0.0;
#pragma unroll
      for (int t = 0; t < n2; ++t) s = fma(T->Wq[t], su[c][e * n2 + t], s);
      sa[c][e] = s;
    }
    __syncthreads();
    // density scaling (eq. euler-pp-density) and the average pressure, once per element
    for (int e = tid; e < EB; e += TH) {
      const double a0 = sa[0][e], a1 = sa[1][e], a2 = sa[2][e], a3 = sa[3][e], a4 = sa[4][e];
      // one reciprocal of the average density: 1/rho-bar for p-bar, and 1/max(rho-bar, eps_rho)
      // (the clamped value, a constant below eps_rho) for the cancellation scale
      const double ira0 = rcp(a0);
      const double ira = a0 > eps_rho ? ira0 : 1.0 / eps_rho;
      const double ma2 = fma(a1, a1, fma(a2, a2, a3 * a3));
      const double pbar = (g - 1.0) * fma(-0.5 * ma2, ira0, a4);
      long long mn = dkey(DBL_MAX);
#pragma unroll
      for (int t = 0; t < n2; ++t) {
        const long long kv = dkey(su[0][e * n2 + t]);
        mn = kv < mn ? kv : mn;
      }
      const double rmin = dkey_inv(mn);
      double th_r = 1.0;
      if (rmin < eps_rho) {
        const double den = a0 - rmin;
        th_r = den > 0.0 ? fmin(1.0, fmax(0.0, (a0 - eps_rho) / den)) : 1.0;
      }
      se[PE_RBAR][e] = a0;
      se[PE_PBAR][e] = pbar;
      se[PE_SA][e] = fma(0.5 * ma2, ira, fabs(a4));
      se[PE_THR][e] = th_r;
      se[PE_MODE][e] = (!(a0 > 0.0) || !(pbar > 0.0) || !isfinite(a0) || !isfinite(pbar)) ? 2.0 : 0.0;
    }
    __syncthreads();
    // nodal pressures after the density scaling, and their cancellation scales
    const double rbar = se[PE_RBAR][el], th_r = se[PE_THR][el];
    double r0 = u[0];
    if (th_r < 1.0) r0 = rbar + th_r * (u[0] - rbar);
    {
      const double m2 = fma(u[1], u[1], fma(u[2], u[2], u[3] * u[3]));
      const double ir0t = rcp(r0);  // nodes are >= eps_rho after the density scaling
      const double ir0 = r0 >= eps_rho ? ir0t : 1.0 / eps_rho;
      st[0][tid] = fma(0.5 * m2, ir0, fabs(u[4]));             // S_p of the node
      st[1][tid] = (g - 1.0) * fma(-0.5 * m2, ir0t, u[4]);     // p of the node
    }
    __syncthreads();
    // floor eps_p (eq. euler-pp-floors), collapse or pressure scaling (eq.
    // euler-pp-pressure, reading R9), once per element
    for (int e = tid; e < EB; e += TH) {
      long long smax = dkey(se[PE_SA][e]), pmn = dkey(DBL_MAX);
#pragma unroll
      for (int t = 0; t < n2; ++t) {
        const long long a = dkey(st[0][e * n2 + t]), b = dkey(st[1][e * n2 + t]);
        smax = a > smax ? a : smax;
        pmn = b < pmn ? b : pmn;
      }
      const double Smax = dkey_inv(smax), pmin = dkey_inv(pmn);
      const double eps_p = fmax(64.0 * eps, 8192.0 * eps * Smax);
      const double rb = se[PE_RBAR][e], pbar = se[PE_PBAR][e], thr = se[PE_THR][e];
      double mode = se[PE_MODE][e], thp = 1.0, trho = 1.0, tall = 1.0;
      if (mode == 0.0) {
        if (rb <= eps_rho || pbar <= eps_p) {  // vacuum-like average: collapse (reading R9)
          mode = 1.0;
          trho = tall = 0.0;
        } else {
          if (thr < 1.0) trho = thr;
          if (pmin < eps_p) {
            const double den = pbar - pmin;
            thp = den > 0.0 ? fmin(1.0, fmax(0.0, (pbar - eps_p) / den)) : 1.0;
            if (thp < 1.0) {
              trho *= thp;
              tall = thp;
            }
          }
        }
      }
      se[PE_MODE][e] = mode;
      se[PE_THP][e] = thp;
      se[PE_TRHO][e] = trho;
      se[PE_TALL][e] = tall;
    }
    __syncthreads();
    const double mode = se[PE_MODE][el];
    if (mode == 2.0) {
      if (q == 0 && valid) atomicOr(status, ST_INADMISSIBLE);
    } else if (mode == 1.0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) u[c] = sa[c][el];
    } else {
      u[0] = r0;
      const double thp = se[PE_THP][el];
      if (thp < 1.0) {
#pragma unroll
        for (int c = 0; c < 5; ++c) u[c] = sa[c][el] + thp * (u[c] - sa[c][el]);
      }
    }
    t_rho = se[PE_TRHO][el];
    t_all = se[PE_TALL][el];
  }
  {
    unsigned act = 0u;
    if (prm.oe_hydro && sD[el][P] < 0.99) act |= ACT_OE_HYDRO;
    if (t_rho < 1.0 || t_all < 1.0) act |= ACT_PP;
    warp_or(prm.activity, act);
  }
  if (frz && q == 0 && valid) {
    double* f = frz + (size_t)k * (n + 2);
#pragma unroll
    for (int l = 0; l < n; ++l) f[l] = prm.oe_hydro ? sD[el][l] : 1.0;
    f[n] = t_rho;
    f[n + 1] = t_all;
  }
  if (valid) {
#pragma unroll
    for (int c = 0; c < 5; ++c) S[MHD_CHK(c * N + (size_t)k * n2 + q, 5 * N)] = u[c];
  }
}

// ---- launchers: hydro stage map -----------------------------------------------------
template <int P>
static void launch_stats(const double* F, size_t stride, int nc, const StatsView& V, const Tab* T, const Mesh& M,
                         cudaStream_t st) {
  size_t total = (size_t)nc * 3 * M.K;
  k_stats<P><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(F, stride, nc, V, T, M);
  dim3 grid(M.nx > M.ny ? M.nx : M.ny, 2);
  k_lines<<<grid, 256, 0, st>>>(nc, V, M);
  k_global<<<1, 256, 0, st>>>(nc, P + 1, V, M);
}

template <int P>
static void stab_hydro_impl(double* S, unsigned* status, const Tab* T, const Mesh& M, const Stab& prm,
                            const double* dtp, double dtfac, double* work, double* frz, cudaStream_t st) {
  StatsView V = stats_view(work, P, M);
  if (prm.oe_hydro) launch_stats<P>(S, (size_t)M.K * (P + 1) * (P + 1), 5, V, T, M, st);
  using C = PCfg<P>;
  k_oe_pp<P><<<(unsigned)((M.K + C::EB - 1) / C::EB), C::threads, 0, st>>>(S, V, T, M, prm, dtp, dtfac, status,
                                                                             frz);
}

// Adjoint of the hydro stage map with its coefficients frozen at the values
// the forward map recorded in frz: lam <- P_OE^T P_PP^T lam, in place.
//   P_PP: U'' = t U* + (1 - t) avg(U*), avg = sum_q (w_q / 4) U*_q
//         -> lam* = t lam'' + (w_q / 4)(1 - t) sum_q' lam''_q'
//   P_OE: U' = Phi diag(D) N Phi^T W U (Legendre modes, quadrature W, norms N)
//         -> lam = W Phi N diag(D) Phi^T lam'
template <int P>
__global__ void __launch_bounds__(OCfg<P>::threads) k_adj_stage_map(double* __restrict__ lam,
                                                                    const double* __restrict__ frz,
                                                                    const Tab* __restrict__ T, Mesh M, int oe,
                                                                    int pp) {
  using C = OCfg<P>;
  constexpr int n = C::n, n2 = C::n2, EB = C::EB, SW = C::SW;
  __shared__ double su[5][EB * SW];
  __shared__ double st[5][EB * SW];
  const size_t N = (size_t)M.K * n2;
  const int tid = threadIdx.x, el = tid / SW, q = tid % SW;
  const bool node = q < n2;
  const int k = blockIdx.x * EB + el;
  const bool valid = k < M.K && node;
  const int kk = k < M.K ? k : M.K - 1;
  const int qq = node ? q : 0;
  const int i = qq % n, j = qq / n;
  const double* f = frz + (size_t)kk * (n + 2);
  double l5[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) l5[c] = node ? lam[c * N + (size_t)kk * n2 + q] : 0.0;
  if (pp) {
    const double wq = node ? 0.25 * T->wp[i] * T->wp[j] : 0.0;
    const int lead = (threadIdx.x & 31) & ~(SW - 1);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const double sum = __shfl_sync(0xffffffffu, seg_sum<SW>(l5[c]), lead);
      const double t = c == 0 ? f[n] : f[n + 1];
      l5[c] = fma(t, l5[c], wq * (1.0 - t) * sum);
    }
  }
  if (oe) {
#pragma unroll
    for (int c = 0; c < 5; ++c) su[c][tid] = l5[c];
    __syncthreads();
    if (node) {  // Vb[b][i] = sum_j P_b(x_j) lam[j][i]   (b = j of this lane)
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double v = 0.0;
#pragma unroll
        for (int jj = 0; jj < n; ++jj) v = fma(T->Leg[jj][j], su[c][el * SW + jj * n + i], v);
        st[c][tid] = v;
      }
    }
    __syncthreads();
    if (node) {  // s[b][a] = N_a N_b D_max(a,b) sum_i P_a(x_i) Vb[b][i]   (a = i, b = j)
      const double fs = T->LegN[i] * T->LegN[j] * f[i > j ? i : j];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double v = 0.0;
#pragma unroll
        for (int ii = 0; ii < n; ++ii) v = fma(T->Leg[ii][i], st[c][el * SW + j * n + ii], v);
        su[c][tid] = fs * v;
      }
    }
    __syncthreads();
    if (node) {  // Tb[b][i] = w_i sum_a P_a(x_i) s[b][a]
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < n; ++a) v = fma(T->Leg[i][a], su[c][el * SW + j * n + a], v);
        st[c][tid] = T->wp[i] * v;
      }
    }
    __syncthreads();
    if (node) {  // lam[j][i] = w_j sum_b P_b(x_j) Tb[b][i]
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double v = 0.0;
#pragma unroll
        for (int b = 0; b < n; ++b) v = fma(T->Leg[j][b], st[c][el * SW + b * n + i], v);
        l5[c] = T->wp[j] * v;
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int c = 0; c < 5; ++c) lam[c * N + (size_t)k * n2 + q] = l5[c];
  }
}

void stab_hydro_adjoint(int p, double* lam, const double* frz, const Tab* T, const Mesh& M, int oe, int pp,
                        cudaStream_t st) {
#define MHD_ADJ_MAP(PP)                                                                                       \
  k_adj_stage_map<PP><<<(unsigned)((M.K + OCfg<PP>::EB - 1) / OCfg<PP>::EB), OCfg<PP>::threads, 0, st>>>( \
      lam, frz, T, M, oe, pp)
  switch (p) {
    case 1: MHD_ADJ_MAP(1); break;
    case 2: MHD_ADJ_MAP(2); break;
    case 3: MHD_ADJ_MAP(3); break;
    case 4: MHD_ADJ_MAP(4); break;
  }
#undef MHD_ADJ_MAP
}

void stab_hydro(int p, double* S, unsigned* status, const Tab* T, const Mesh& M, const Stab& prm, const double* dtp,
                double dtfac, double* work, double* frz, cudaStream_t st) {
  switch (p) {
    case 1: stab_hydro_impl<1>(S, status, T, M, prm, dtp, dtfac, work, frz, st); break;
    case 2: stab_hydro_impl<2>(S, status, T, M, prm, dtp, dtfac, work, frz, st); break;
    case 3: stab_hydro_impl<3>(S, status, T, M, prm, dtp, dtfac, work, frz, st); break;
    case 4: stab_hydro_impl<4>(S, status, T, M, prm, dtp, dtfac, work, frz, st); break;
  }
}

// ============================ artificial resistivity =============================
// B closure helpers (element-blocked owned DOFs, see mhd_internal.cuh).
template <int KM>
__device__ __forceinline__ double bx_cl(const double* Bx, int ex, int ey, int a, int b, const Mesh& M) {
  constexpr int mm = KM + 1, mL = KM + 2;
  const size_t Z = (size_t)M.K * mm * mm;
  if (a == mL - 1) return Bx[MHD_CHK(((size_t)ey * M.nx + wrap(ex + 1, M.nx)) * mm * mm + b * mm, Z)];
  return Bx[MHD_CHK(((size_t)ey * M.nx + ex) * mm * mm + b * mm + a, Z)];
}
template <int KM>
__device__ __forceinline__ double by_cl(const double* By, int ex, int ey, int a, int b, const Mesh& M) {
  constexpr int mm = KM + 1, mL = KM + 2;
  const size_t Z = (size_t)M.K * mm * mm;
  if (b == mL - 1) return By[MHD_CHK(((size_t)wrap(ey + 1, M.ny) * M.nx + ex) * mm * mm + a, Z)];
  return By[MHD_CHK(((size_t)ey * M.nx + ex) * mm * mm + b * mm + a, Z)];
}

// Component d of B_h of element (ex, ey) at reference point (x, y) given as 1D
// basis values: LX = l^L(x) [mL], GX = g(x) [mm], MX = l^M(x) [mm], likewise Y.
template <int KM>
__device__ double B_eval(const double* B, size_t Z, int d, int ex, int ey, const double* LX, const double* GX,
                         const double* MX, const double* LY, const double* GY, const double* MY, const Mesh& M) {
  constexpr int mm = KM + 1, mL = KM + 2;
  double v = 0.0;
  if (d == 0) {
    for (int b = 0; b < mm; ++b) {
      double row = 0.0;
      for (int a = 0; a < mL; ++a) row = fma(LX[a], bx_cl<KM>(B, ex, ey, a, b, M), row);
      v = fma(GY[b], row, v);
    }
  } else if (d == 1) {
    for (int b = 0; b < mL; ++b) {
      double row = 0.0;
      for (int a = 0; a < mm; ++a) row = fma(GX[a], by_cl<KM>(B + Z, ex, ey, a, b, M), row);
      v = fma(LY[b], row, v);
    }
  } else {
    const double* Bz = B + 2 * Z + ((size_t)ey * M.nx + ex) * mm * mm;
    for (int b = 0; b < mm; ++b) {
      double row = 0.0;
      for (int a = 0; a < mm; ++a) row = fma(MX[a], Bz[b * mm + a], row);
      v = fma(MY[b], row, v);
    }
  }
  return v;
}

// Per element: exact integrals of Bx, By, Bz (global means), max/min of the
// owned DOFs, the tangential jump measures J_0 of the -x face (B_y, B_z) and
// the -y face (B_x, B_z), and the directional speeds a_{I,K}.
// ar[K][16]: 0-2 integrals, 3-5 max, 6-8 min, 9-10 -x face (By, Bz), 11-12 -y face (Bx, Bz), 13-14 a_x, a_y
template <int P, int KM>
__global__ void k_ar_elem(const double* __restrict__ rho, const double* __restrict__ Y, const double* __restrict__ B,
                          const Tab* __restrict__ T, Mesh M, double* __restrict__ ar) {
  constexpr int n = P + 1, n2 = n * n, mm = KM + 1, mL = KM + 2, q2 = KM + 2;
  // node families that coincide with the DG nodes (the same GLL rule, so the
  // same doubles): GLL(k+1) at k = p - 1, GLL(k) at k = p; the interpolation
  // between them is exactly the identity and is skipped (same bits)
  constexpr bool LID = mL == n, MID = mm == n;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.K) return;
  const size_t Z = (size_t)M.K * mm * mm, N = (size_t)M.K * n2;
  const int ex = k % M.nx, ey = k / M.nx;
  // this element's closures: Bx [b < mm][a < mL], By [b < mL][a < mm], Bz [b][a]
  double bx[mm][mL], by[mL][mm], bz[mm][mm];
#pragma unroll
  for (int b = 0; b < mm; ++b)
#pragma unroll
    for (int a = 0; a < mL; ++a) bx[b][a] = bx_cl<KM>(B, ex, ey, a, b, M);
#pragma unroll
  for (int b = 0; b < mL; ++b)
#pragma unroll
    for (int a = 0; a < mm; ++a) by[b][a] = by_cl<KM>(B + Z, ex, ey, a, b, M);
#pragma unroll
  for (int b = 0; b < mm; ++b)
#pragma unroll
    for (int a = 0; a < mm; ++a) bz[b][a] = B[MHD_CHK(2 * Z + (size_t)k * mm * mm + b * mm + a, 3 * Z)];
  double out[16];
  // exact element integrals: the integral of a nodal basis function is its
  // quadrature weight, so the weight rows in place of the interpolation rows
  // give the integral over the reference element (x-pass, then y-pass)
  {
    double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
    for (int b = 0; b < mm; ++b) {
      double row = 0.0;
#pragma unroll
      for (int a = 0; a < mL; ++a) row = fma(T->wL[a], bx[b][a], row);
      sx = fma(T->wG[b], row, sx);
    }
#pragma unroll
    for (int b = 0; b < mL; ++b) {
      double row = 0.0;
#pragma unroll
      for (int a = 0; a < mm; ++a) row = fma(T->wG[a], by[b][a], row);
      sy = fma(T->wL[b], row, sy);
    }
#pragma unroll
    for (int b = 0; b < mm; ++b) {
      double row = 0.0;
#pragma unroll
      for (int a = 0; a < mm; ++a) row = fma(T->wM[a], bz[b][a], row);
      sz = fma(T->wM[b], row, sz);
    }
    out[0] = M.Jdet * sx; out[1] = M.Jdet * sy; out[2] = M.Jdet * sz;
  }
  for (int d = 0; d < 3; ++d) {
    double mx = -DBL_MAX, mn = DBL_MAX;
    const double* A = B + d * Z + (size_t)k * mm * mm;
    for (int t = 0; t < mm * mm; ++t) { mx = fmax(mx, A[t]); mn = fmin(mn, A[t]); }
    out[3 + d] = mx; out[6 + d] = mn;
  }
  // tangential jumps on the lower faces, Gauss(k+2) face rule (reading R6):
  // each trace collapses the normal direction once, then is evaluated at the
  // face points
  {  // x-face (I = 0): B_y and B_z of this element at x = -1 and of the -x neighbour at x = +1
    const int exA = wrap(ex - 1, M.nx);
    double ryB[mL], ryA[mL], rzB[mm], rzA[mm];
#pragma unroll
    for (int b = 0; b < mL; ++b) {
      double vB = 0.0, vA = 0.0;
#pragma unroll
      for (int a = 0; a < mm; ++a) {
        vB = fma(T->G_end[0][a], by[b][a], vB);
        vA = fma(T->G_end[1][a], by_cl<KM>(B + Z, exA, ey, a, b, M), vA);
      }
      ryB[b] = vB; ryA[b] = vA;
    }
    const double* bzA = B + 2 * Z + ((size_t)ey * M.nx + exA) * mm * mm;
#pragma unroll
    for (int b = 0; b < mm; ++b) {
      double vB = 0.0, vA = 0.0;
#pragma unroll
      for (int a = 0; a < mm; ++a) {
        vB = fma(T->M_end[0][a], bz[b][a], vB);
        vA = fma(T->M_end[1][a], bzA[b * mm + a], vA);
      }
      rzB[b] = vB; rzA[b] = vA;
    }
    double accy = 0.0, accz = 0.0;
#pragma unroll
    for (int t = 0; t < q2; ++t) {
      double yB = 0.0, yA = 0.0, zB = 0.0, zA = 0.0;
#pragma unroll
      for (int b = 0; b < mL; ++b) { yB = fma(T->L_2[t][b], ryB[b], yB); yA = fma(T->L_2[t][b], ryA[b], yA); }
#pragma unroll
      for (int b = 0; b < mm; ++b) { zB = fma(T->M_2[t][b], rzB[b], zB); zA = fma(T->M_2[t][b], rzA[b], zA); }
      const double jy = yB - yA, jz = zB - zA;
      accy = fma(0.5 * T->w2[t] * jy, jy, accy);
      accz = fma(0.5 * T->w2[t] * jz, jz, accz);
    }
    out[9] = fsqrt(accy); out[10] = fsqrt(accz);
  }
  {  // y-face (I = 1): B_x and B_z of this element at y = -1 and of the -y neighbour at y = +1
    const int eyA = wrap(ey - 1, M.ny);
    double cxB[mL], cxA[mL], czB[mm], czA[mm];
#pragma unroll
    for (int a = 0; a < mL; ++a) {
      double vB = 0.0, vA = 0.0;
#pragma unroll
      for (int b = 0; b < mm; ++b) {
        vB = fma(T->G_end[0][b], bx[b][a], vB);
        vA = fma(T->G_end[1][b], bx_cl<KM>(B, ex, eyA, a, b, M), vA);
      }
      cxB[a] = vB; cxA[a] = vA;
    }
    const double* bzA = B + 2 * Z + ((size_t)eyA * M.nx + ex) * mm * mm;
#pragma unroll
    for (int a = 0; a < mm; ++a) {
      double vB = 0.0, vA = 0.0;
#pragma unroll
      for (int b = 0; b < mm; ++b) {
        vB = fma(T->M_end[0][b], bz[b][a], vB);
        vA = fma(T->M_end[1][b], bzA[b * mm + a], vA);
      }
      czB[a] = vB; czA[a] = vA;
    }
    double accx = 0.0, accz = 0.0;
#pragma unroll
    for (int t = 0; t < q2; ++t) {
      double xB = 0.0, xA = 0.0, zB = 0.0, zA = 0.0;
#pragma unroll
      for (int a = 0; a < mL; ++a) { xB = fma(T->L_2[t][a], cxB[a], xB); xA = fma(T->L_2[t][a], cxA[a], xA); }
#pragma unroll
      for (int a = 0; a < mm; ++a) { zB = fma(T->M_2[t][a], czB[a], zB); zA = fma(T->M_2[t][a], czA[a], zA); }
      const double jx = xB - xA, jz = zB - zA;
      accx = fma(0.5 * T->w2[t] * jx, jx, accx);
      accz = fma(0.5 * T->w2[t] * jz, jz, accz);
    }
    out[11] = fsqrt(accx); out[12] = fsqrt(accz);
  }
  // a_{I,K} = max over DG nodes of |u_I| + |B_h| / sqrt(rho): B at the nodes
  // sum-factorised (x-pass, then y-pass: the order of the single-point tensor
  // evaluation), one component at a time
  double b2[n2];
#pragma unroll
  for (int q = 0; q < n2; ++q) b2[q] = 0.0;
  {
    double tx[mm][n];
#pragma unroll
    for (int b = 0; b < mm; ++b)
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double v = 0.0;
        if constexpr (LID) v = bx[b][i];
        else {
#pragma unroll
          for (int a = 0; a < mL; ++a) v = fma(T->L_P[i][a], bx[b][a], v);
        }
        tx[b][i] = v;
      }
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double v = 0.0;
#pragma unroll
        for (int b = 0; b < mm; ++b) v = fma(T->G_P[j][b], tx[b][i], v);
        b2[j * n + i] = v * v;
      }
  }
  if constexpr (LID) {  // By rows to the DG x-nodes; GLL(k+1) y is the DG rule (copy)
    double ty[mL][n];
#pragma unroll
    for (int b = 0; b < mL; ++b)
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < mm; ++a) v = fma(T->G_P[i][a], by[b][a], v);
        ty[b][i] = v;
      }
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int i = 0; i < n; ++i) b2[j * n + i] = fma(ty[j][i], ty[j][i], b2[j * n + i]);
  } else {  // By columns to the DG y-nodes, then the x-pass (the cheaper order)
    double tc[mm][n];
#pragma unroll
    for (int a = 0; a < mm; ++a)
#pragma unroll
      for (int j = 0; j < n; ++j) {
        double v = 0.0;
#pragma unroll
        for (int b = 0; b < mL; ++b) v = fma(T->L_P[j][b], by[b][a], v);
        tc[a][j] = v;
      }
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < mm; ++a) v = fma(T->G_P[i][a], tc[a][j], v);
        b2[j * n + i] = fma(v, v, b2[j * n + i]);
      }
  }
  {
    double tz[mm][n];
#pragma unroll
    for (int b = 0; b < mm; ++b)
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double v = 0.0;
        if constexpr (MID) v = bz[b][i];
        else {
#pragma unroll
          for (int a = 0; a < mm; ++a) v = fma(T->M_P[i][a], bz[b][a], v);
        }
        tz[b][i] = v;
      }
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double v = 0.0;
        if constexpr (MID) v = tz[j][i];
        else {
#pragma unroll
          for (int b = 0; b < mm; ++b) v = fma(T->M_P[j][b], tz[b][i], v);
        }
        b2[j * n + i] = fma(v, v, b2[j * n + i]);
      }
  }
  double ax = 0.0, ay = 0.0;
#pragma unroll
  for (int q = 0; q < n2; ++q) {
    const size_t gq = MHD_CHK((size_t)k * n2 + q, N);
    const double va = fsqrt(b2[q] * rcp(rho[gq]));  // |B_h| / sqrt(rho)
    ax = fmax(ax, fabs(Y[N + gq]) + va);
    ay = fmax(ay, fabs(Y[2 * N + gq]) + va);
  }
  out[13] = ax; out[14] = ay; out[15] = 0.0;
  for (int c = 0; c < 16; ++c) ar[(size_t)k * 16 + c] = out[c];
}

// Global reduction of the A.R. partials in two fixed-order levels: k_ar_part
// reduces 256-element chunks (one block each), k_ar_global the chunk results.
__device__ __forceinline__ void ar_combine(double* x, const double* y) {
  for (int c = 0; c < 3; ++c) x[c] += y[c];
  for (int c = 3; c < 6; ++c) x[c] = fmax(x[c], y[c]);
  for (int c = 6; c < 9; ++c) x[c] = fmin(x[c], y[c]);
}

__device__ void ar_block_reduce(double acc[9], double (*sm)[9]) {
  for (int c = 0; c < 9; ++c) sm[threadIdx.x][c] = acc[c];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) ar_combine(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
}

__global__ void k_ar_part(const double* __restrict__ ar, Mesh M, double* __restrict__ part) {
  __shared__ double sm[256][9];
  double acc[9] = {0, 0, 0, -DBL_MAX, -DBL_MAX, -DBL_MAX, DBL_MAX, DBL_MAX, DBL_MAX};
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < M.K) {
    const double* a = ar + (size_t)k * 16;
    for (int c = 0; c < 9; ++c) acc[c] = a[c];
  }
  ar_block_reduce(acc, sm);
  if (threadIdx.x == 0)
    for (int c = 0; c < 9; ++c) part[(size_t)blockIdx.x * 9 + c] = sm[0][c];
}

__global__ void k_ar_global(const double* __restrict__ part, int nparts, Mesh M, double* __restrict__ g) {
  __shared__ double sm[256][9];
  double acc[9] = {0, 0, 0, -DBL_MAX, -DBL_MAX, -DBL_MAX, DBL_MAX, DBL_MAX, DBL_MAX};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) ar_combine(acc, part + (size_t)b * 9);
  ar_block_reduce(acc, sm);
  if (threadIdx.x == 0) {
    double area = M.K * 4.0 * M.Jdet;
    double amp[3], linf[3];
    for (int d = 0; d < 3; ++d) {
      double mean = sm[0][d] / area;
      amp[d] = fmax(sm[0][3 + d] - mean, mean - sm[0][6 + d]);
      linf[d] = fmax(fabs(sm[0][3 + d]), fabs(sm[0][6 + d]));
    }
    // Delta^B_I over T_x = {y, z}, T_y = {x, z}; roundoff-constant directions off (reading R8)
    double Dx = fmax(amp[1], amp[2]), Dy = fmax(amp[0], amp[2]);
    g[0] = Dx; g[1] = Dy;
    g[2] = Dx <= 1024.0 * DBL_EPSILON * fmax(fmax(linf[1], linf[2]), 1e-300) ? 1.0 : 0.0;
    g[3] = Dy <= 1024.0 * DBL_EPSILON * fmax(fmax(linf[0], linf[2]), 1e-300) ? 1.0 : 0.0;
  }
}

// eta_K = C_eta max_I h_I a_I R_I / (2p+1), R_I = min(C_s sigma^B_I, 1).
__global__ void k_ar_eta(const double* __restrict__ ar, const double* __restrict__ g, Mesh M, Stab prm, int p,
                         double* __restrict__ eta) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.K) return;
  const int ex = k % M.nx, ey = k / M.nx;
  const int kE = ey * M.nx + wrap(ex + 1, M.nx), kN = wrap(ey + 1, M.ny) * M.nx + ex;
  const double* a = ar + (size_t)k * 16;
  double e = 0.0;
  for (int I = 0; I < 2; ++I) {
    double sig = 0.0;
    if (g[2 + I] == 0.0) {
      const double* b = ar + (size_t)(I == 0 ? kE : kN) * 16;
      for (int tc = 0; tc < 2; ++tc) {
        double J0 = a[9 + 2 * I + tc] + b[9 + 2 * I + tc];
        sig = fmax(sig, J0 / (2.0 * g[I]));
      }
    }
    double R = fmin(prm.C_s * sig, 1.0);
    double h = I == 0 ? M.hx : M.hy;
    e = fmax(e, h / (2.0 * p + 1.0) * a[13 + I] * R);
  }
  eta[k] = prm.C_eta * e;
  warp_or(prm.activity, prm.C_eta * e > 0.0 ? ACT_AR : 0u);
}

void stab_eta(int p, int k, const double* rho, const double* Y, const double* B, const Tab* T, const Mesh& M,
              const Stab& prm, double* eta, double* work, cudaStream_t st) {
  StatsView V = stats_view(work, p, M);
  double* ar = V.jx;  // the A.R. partials reuse the sensor area: [K][16] <= 2 * 5 * n * K
  double* g = V.glob;
  unsigned bl = (unsigned)((M.K + 127) / 128);
#define MHD_AR_CASE(PP, KK) k_ar_elem<PP, KK><<<bl, 128, 0, st>>>(rho, Y, B, T, M, ar)
  MHD_DISPATCH_PK(p, k, MHD_AR_CASE);
#undef MHD_AR_CASE
  const int nparts = (M.K + 255) / 256;
  double* part = V.part;
  k_ar_part<<<nparts, 256, 0, st>>>(ar, M, part);
  k_ar_global<<<1, 256, 0, st>>>(part, nparts, M, g);
  k_ar_eta<<<bl, 128, 0, st>>>(ar, g, M, prm, p, eta);
}

// ============================ velocity OE ==========================================
// Psi = Phi L^{-T} per element (n2 x n2, row q = node, column alpha = basis in
// shell order), G = Phi^T W Phi = L L^T.  One thread per element (32 elements per
// block); the Gram matrix is sum-factorised,
//   G[(a,b),(a',b')] = sum_j P_b(x_j) P_b'(x_j) H_j[a][a'],
//   H_j[a][a'] = sum_i W_ij P_a(x_i) P_a'(x_i),
// and L is kept in shared memory laid out element-innermost.
template <int P>
struct VPrep {
  static constexpr int n = P + 1, n2 = n * n, NL = n2 * (n2 + 1) / 2, NA = n * (n + 1) / 2, NH = n * NA;
  static constexpr int SIZE = NL + NH;
};

__device__ __forceinline__ int tri(int r, int c) { return r * (r + 1) / 2 + c; }  // c <= r

template <int P>
__global__ void __launch_bounds__(32) k_vel_prep(const double* __restrict__ rho, double* __restrict__ Psi,
                                                 const Tab* __restrict__ T, Mesh M) {
  using V = VPrep<P>;
  constexpr int n = V::n, n2 = V::n2;
  extern __shared__ double smp[];
  const int lane = threadIdx.x;
  const int k = blockIdx.x * 32 + lane;
  const int kk = k < M.K ? k : M.K - 1;
#define LS(idx) smp[(size_t)(idx) * 32 + lane]
#define HS(idx) smp[(size_t)(V::NL + (idx)) * 32 + lane]
  // shell-ordered Legendre index pairs (a, b) of the basis: shell l = max(a, b) holds [l^2, (l+1)^2)
  int ia[n2], ib[n2];
  {
    int t = 0;
#pragma unroll
    for (int l = 0; l <= P; ++l)
#pragma unroll
      for (int b = 0; b <= l; ++b)
#pragma unroll
        for (int a = 0; a <= l; ++a)
          if ((a > b ? a : b) == l) { ia[t] = a; ib[t] = b; ++t; }
  }
  double W[n2];
#pragma unroll
  for (int q = 0; q < n2; ++q) W[q] = M.Jdet * T->wp[q % n] * T->wp[q / n] * rho[(size_t)kk * n2 + q];
#pragma unroll
  for (int j = 0; j < n; ++j)
#pragma unroll
    for (int a = 0; a < n; ++a)
#pragma unroll
      for (int a2 = 0; a2 <= a; ++a2) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < n; ++i) s = fma(W[j * n + i], T->LegLeg[i][a][a2], s);
        HS(j * V::NA + tri(a, a2)) = s;
      }
#pragma unroll
  for (int al = 0; al < n2; ++al)
#pragma unroll
    for (int be = 0; be <= al; ++be) {
      const int a = ia[al], b = ib[al], a2 = ia[be], b2 = ib[be];
      const int pa = a >= a2 ? tri(a, a2) : tri(a2, a);
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < n; ++j) s = fma(T->LegLeg[j][b][b2], HS(j * V::NA + pa), s);
      LS(tri(al, be)) = s;
    }
  // Cholesky G = L L^T in place (row by row)
  double rdiag[n2];
#pragma unroll
  for (int r = 0; r < n2; ++r) {
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      double s = LS(tri(r, c));
#pragma unroll
      for (int t = 0; t < c; ++t) s = fma(-LS(tri(r, t)), LS(tri(c, t)), s);
      if (r == c) {
        const double d = fsqrt(s);
        LS(tri(r, r)) = d;
        rdiag[r] = rcp(d);
      } else {
        LS(tri(r, c)) = s * rdiag[c];
      }
    }
  }
  // rows of Psi: psi_q L^T = phi_q (forward substitution)
  double* out = Psi + (size_t)kk * n2 * n2;
#pragma unroll 1
  for (int q = 0; q < n2; ++q) {
    double row[n2];
#pragma unroll
    for (int al = 0; al < n2; ++al) {
      double s = T->Phi[q][al];
#pragma unroll
      for (int b = 0; b < al; ++b) s = fma(-row[b], LS(tri(al, b)), s);
      row[al] = s * rdiag[al];
    }
    if (k < M.K) {
#pragma unroll
      for (int al = 0; al < n2; ++al) out[q * n2 + al] = row[al];
    }
  }
#undef LS
#undef HS
}

template <int P>
static void launch_vel_prep(const double* rho, double* chol, const Tab* T, const Mesh& M, cudaStream_t st) {
  const size_t smem = sizeof(double) * VPrep<P>::SIZE * 32;
  k_vel_prep<P><<<(unsigned)((M.K + 31) / 32), 32, smem, st>>>(rho, chol, T, M);
}

// Opt-in dynamic shared memory of the velocity-projector kernel (context creation).
cudaError_t stab_prepare(int p) {
  switch (p) {
    case 1: return cudaFuncSetAttribute((const void*)k_vel_prep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * VPrep<1>::SIZE * 32));
    case 2: return cudaFuncSetAttribute((const void*)k_vel_prep<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * VPrep<2>::SIZE * 32));
    case 3: return cudaFuncSetAttribute((const void*)k_vel_prep<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * VPrep<3>::SIZE * 32));
    case 4: return cudaFuncSetAttribute((const void*)k_vel_prep<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * VPrep<4>::SIZE * 32));
    default: return cudaErrorInvalidValue;
  }
}

void stab_vel_prep(int p, const double* rho, double* chol, const Tab* T, const Mesh& M, cudaStream_t st) {
  switch (p) {
    case 1: launch_vel_prep<1>(rho, chol, T, M, st); break;
    case 2: launch_vel_prep<2>(rho, chol, T, M, st); break;
    case 3: launch_vel_prep<3>(rho, chol, T, M, st); break;
    case 4: launch_vel_prep<4>(rho, chol, T, M, st); break;
  }
}

// Velocity OE map with heating of e.  One thread per node (EB elements x
// (p+1)^2 threads, no padding); B at the DG nodes is sum-factorised over the
// block (an x-pass of the closures, then a y-pass, in the order of the
// single-point evaluation B_eval, so the values are the same bit for bit); the
// rate, the sensor and the factors are computed once per element or per
// (element, direction, order) in flat item loops, as in k_oe_pp.
// frz (may be null): the damping factors D_0..D_p of every element, [K][p+1],
// for the adjoint (frozen coefficients).
template <int P>
struct VCfg {
  static constexpr int n = P + 1, n2 = n * n;
  static constexpr int EB = P == 1 ? 64 : P == 2 ? 28 : P == 3 ? 8 : 4;
  static constexpr int threads = EB * n2;
};

template <int P, int KM, bool R2 = false>
__global__ void __launch_bounds__(VCfg<P>::threads) k_vel_oe(const double* __restrict__ rho, double* __restrict__ Y,
                                                             const double* __restrict__ B,
                                                             const double* __restrict__ Psi, StatsView V,
                                                             const Tab* __restrict__ T, Mesh M, Stab prm,
                                                             const double* __restrict__ dtp, double dtfac,
                                                             double* __restrict__ frz) {
  using C = VCfg<P>;
  constexpr int n = C::n, n2 = C::n2, EB = C::EB, TH = C::threads;
  constexpr int mm = KM + 1, mL = KM + 2;
  // node families equal to the DG nodes (GLL(k+1) at k = p - 1, GLL(k) at
  // k = p): their interpolation to the DG nodes is the identity, skipped
  constexpr bool LID = mL == n, MID = mm == n;
  // 2D2V (R2): u_z = B_z = 0, so only u_x, u_y are filtered (u_z stays 0)
  constexpr int ND = R2 ? 2 : 3;
  __shared__ double sPsi[EB][n2 * n2];
  __shared__ double sWu[3][EB * n2];
  __shared__ double sc[3][EB * n2];
  // closures of Bx, By and Bz, and the x-passes; one pad double per element so
  // that the element-fastest x-pass items do not collide in banks
  __shared__ double sB[EB][mm * mL + mL * mm + mm * mm + 1];
  __shared__ double sT[EB][mm * n + mL * n + mm * n + 1];
  __shared__ double sax[2][EB * n2];                       // |u_I| + |B|/sqrt(rho) per node
  __shared__ double ssig[EB][2 * n];
  __shared__ double sD[EB][n];
  __shared__ double sH[EB][n];                             // (1 - D_l^2) / 2: heating factor of shell l
  __shared__ double slam[EB][2];
  __shared__ double sMw[n2];                               // Jdet w_i w_j of the DG nodes
  const size_t N = (size_t)M.K * n2, Z = (size_t)M.K * mm * mm;
  const int tid = threadIdx.x, el = tid / n2, q = tid % n2;
  const int k0 = blockIdx.x * EB;
  const int k = k0 + el;
  const bool valid = k < M.K;
  const int kk = valid ? k : M.K - 1;
  const int i = q % n, j = q / n;
  double u[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < ND; ++d) u[d] = Y[MHD_CHK((1 + d) * N + (size_t)kk * n2 + q, 4 * N)];
  const double r_ = rho[MHD_CHK((size_t)kk * n2 + q, N)];
  {  // Psi of the element to shared memory as asynchronous copies (cp.async), waited
     // for only where the projections need it, so that the B evaluation and the
     // sensor run meanwhile
    const double* src = Psi + MHD_CHK((size_t)kk * n2 * n2, (size_t)M.K * n2 * n2);
    for (int t = q; t < n2 * n2; t += n2) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(&sPsi[el][t]);
      const size_t gsrc = __cvta_generic_to_global(src + t);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gsrc) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if (tid < n2) sMw[tid] = M.Jdet * T->wp[tid % n] * T->wp[tid / n];
  // closures of B (Bx [b < mm][a < mL], By [b < mL][a < mm], Bz [b][a]) of the block's elements
  constexpr int NB = mm * mL + mL * mm + (R2 ? 0 : mm * mm);
  for (int it = tid; it < EB * NB; it += TH) {
    const int e = it / NB, w = it % NB;
    const int ke = min(k0 + e, M.K - 1), ex = ke % M.nx, ey = ke / M.nx;
    double v;
    if (w < mm * mL) v = bx_cl<KM>(B, ex, ey, w % mL, w / mL, M);
    else if (w < 2 * mm * mL) { const int r = w - mm * mL; v = by_cl<KM>(B + Z, ex, ey, r % mm, r / mm, M); }
    else v = B[MHD_CHK(2 * Z + (size_t)ke * mm * mm + (w - 2 * mm * mL), 3 * Z)];
    sB[e][w] = v;
  }
  __syncthreads();
  // first passes: Bx rows (Gauss y) to the DG x-nodes; By (Gauss x, GLL(k+1) y) columns to
  // the DG y-nodes, the cheaper order (at k = p - 1, where GLL(k+1) y is the DG rule, its rows
  // to the DG x-nodes instead, the y-pass being a copy); Bz rows (GLL(k) y) to the DG x-nodes.
  // Items element-fastest, so that a warp's items come from one family (one branch)
  constexpr int NBY = LID ? mL * n : mm * n;
  constexpr int NT = mm * n + NBY + (R2 ? 0 : mm * n);
  for (int it = tid; it < EB * NT; it += TH) {
    const int e = it % EB, w = it / EB;
    double v = 0.0;
    if (w < mm * n) {
      const int b = w / n, ii = w % n;
      if constexpr (LID) v = sB[e][b * mL + ii];
      else {
#pragma unroll
        for (int a = 0; a < mL; ++a) v = fma(T->L_P[ii][a], sB[e][b * mL + a], v);
      }
    } else if (w < mm * n + NBY) {
      const int r = w - mm * n;
      if constexpr (LID) {  // By rows b to the DG x-nodes
        const int b = r / n, ii = r % n;
#pragma unroll
        for (int a = 0; a < mm; ++a) v = fma(T->G_P[ii][a], sB[e][mm * mL + b * mm + a], v);
      } else {  // By columns a to the DG y-nodes jj
        const int a = r / n, jj = r % n;
#pragma unroll
        for (int b = 0; b < mL; ++b) v = fma(T->L_P[jj][b], sB[e][mm * mL + b * mm + a], v);
      }
    } else {
      const int r = w - mm * n - NBY, b = r / n, ii = r % n;
      if constexpr (MID) v = sB[e][2 * mm * mL + b * mm + ii];
      else {
#pragma unroll
        for (int a = 0; a < mm; ++a) v = fma(T->M_P[ii][a], sB[e][2 * mm * mL + b * mm + a], v);
      }
    }
    sT[e][w] = v;
  }
  __syncthreads();
  {  // y-passes at this node, |B_h| / sqrt(rho) (eq. magnetic-oe-rate)
    double bx = 0.0, by = 0.0, bz = 0.0;
#pragma unroll
    for (int b = 0; b < mm; ++b) bx = fma(T->G_P[j][b], sT[el][b * n + i], bx);
    if constexpr (LID) by = sT[el][mm * n + j * n + i];
    else {  // x-pass of the By columns at DG row j
#pragma unroll
      for (int a = 0; a < mm; ++a) by = fma(T->G_P[i][a], sT[el][mm * n + a * n + j], by);
    }
    if constexpr (!R2) {
      if constexpr (MID) bz = sT[el][mm * n + NBY + j * n + i];
      else {
#pragma unroll
        for (int b = 0; b < mm; ++b) bz = fma(T->M_P[j][b], sT[el][mm * n + NBY + b * n + i], bz);
      }
    }
    const double va = fsqrt(fma(bx, bx, fma(by, by, bz * bz)) * rcp(r_));
    sax[0][tid] = fabs(u[0]) + va;
    sax[1][tid] = fabs(u[1]) + va;
  }
  const double W = sMw[q] * r_;
#pragma unroll
  for (int d = 0; d < ND; ++d) sWu[d][tid] = W * u[d];
  __syncthreads();
  // rate lambda_M,I (eq. magnetic-oe-rate): nodal maxima (integer keys), once per element
  for (int it = tid; it < EB * 2; it += TH) {
    const int e = it / 2, I = it % 2;
    long long mx = dkey(0.0);
#pragma unroll
    for (int t = 0; t < n2; ++t) {
      const long long kv = dkey(sax[I][e * n2 + t]);
      mx = kv > mx ? kv : mx;
    }
    slam[e][I] = (2.0 * P + 1.0) * (I == 0 ? M.ihx : M.ihy) * dkey_inv(mx);
  }
  // sigma_{r,I} (eq. magnetic-oe-sensor), once per (element, direction, order)
  const int Lmax = M.nx > M.ny ? M.nx : M.ny;
  for (int it = tid; it < EB * 2 * n; it += TH) {
    const int e = it / (2 * n), w = it % (2 * n), I = w / n, r = w % n;
    const int ke = min(k0 + e, M.K - 1), ex = ke % M.nx, ey = ke / M.nx;
    const double iDelta = V.lineD[I * Lmax + (I == 0 ? ey : ex)];
    const int kB = I == 0 ? ey * M.nx + wrap(ex + 1, M.nx) : wrap(ey + 1, M.ny) * M.nx + ex;
    ssig[e][w] = sigma_rI(V, ND, n, I, r, ke, kB, iDelta, M.K);
  }
  __syncthreads();
  // D_l = exp(-s_M tau Theta_l) (eq. magnetic-oe-factor), once per (element, shell)
  const double s_tau = prm.s_M * dtp[0] * dtfac;
  for (int it = tid; it < EB * n; it += TH) {
    const int e = it / n, l = it % n;
    double Theta = 0.0;
    for (int I = 0; I < 2; ++I) {
      double ss = 0.0;
      for (int r = 0; r <= l; ++r) ss += ssig[e][I * n + r];
      Theta = fma(slam[e][I], ss, Theta);
    }
    const double Dl = l == 0 ? 1.0 : exp(-s_tau * Theta);
    sD[e][l] = Dl;
    sH[e][l] = 0.5 * (1.0 - Dl * Dl);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // this thread's Psi copies
  __syncthreads();                                         // and everyone else's
  if (frz && q < n && valid) frz[(size_t)k * n + q] = sD[el][q];
  warp_or(prm.activity, sD[el][P] < 0.99 ? ACT_OE_VEL : 0u);
  // coefficients c_alpha = sum_t Psi[t][alpha] W_t u_t (thread q plays alpha)
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < n2; ++t) s = fma(sPsi[el][t * n2 + q], sWu[d][el * n2 + t], s);
    sc[d][tid] = s;
  }
  __syncthreads();
  if (valid) {
    double de = 0.0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      double unew = 0.0;
#pragma unroll
      for (int l = 0; l <= P; ++l) {  // shell l holds basis indices [l^2, (l+1)^2)
        double wl = 0.0;
#pragma unroll
        for (int al = l * l; al < (l + 1) * (l + 1); ++al) wl = fma(sc[d][el * n2 + al], sPsi[el][q * n2 + al], wl);
        unew = fma(sD[el][l], wl, unew);
        if (l > 0) de = fma(sH[el][l] * wl, wl, de);
      }
      Y[MHD_CHK((1 + d) * N + (size_t)k * n2 + q, 4 * N)] = unew;
    }
    Y[MHD_CHK((size_t)k * n2 + q, N)] += de;
  }
}

void stab_vel(int p, int k, const double* rho, double* Y, const double* B, const double* chol, const Tab* T,
              const Mesh& M, const Stab& prm, const double* dtp, double dtfac, double* work, double* frz,
              cudaStream_t st) {
  StatsView V = stats_view(work, p, M);
  const size_t N = (size_t)M.K * (p + 1) * (p + 1);
  const int nc = prm.reduced ? 2 : 3;  // 2D2V: u_z = 0 is constant and never enters the sensor
  switch (p) {
    case 1: launch_stats<1>(Y + N, N, nc, V, T, M, st); break;
    case 2: launch_stats<2>(Y + N, N, nc, V, T, M, st); break;
    case 3: launch_stats<3>(Y + N, N, nc, V, T, M, st); break;
    case 4: launch_stats<4>(Y + N, N, nc, V, T, M, st); break;
  }
#define MHD_VOE_CASE(PP, KK)                                                                                    \
  if (prm.reduced)                                                                                             \
    k_vel_oe<PP, KK, true><<<(unsigned)((M.K + VCfg<PP>::EB - 1) / VCfg<PP>::EB), VCfg<PP>::threads, 0, st>>>( \
        rho, Y, B, chol, V, T, M, prm, dtp, dtfac, frz);                                                        \
  else                                                                                                         \
    k_vel_oe<PP, KK><<<(unsigned)((M.K + VCfg<PP>::EB - 1) / VCfg<PP>::EB), VCfg<PP>::threads, 0, st>>>(       \
        rho, Y, B, chol, V, T, M, prm, dtp, dtfac, frz)
  MHD_DISPATCH_PK(p, k, MHD_VOE_CASE);
#undef MHD_VOE_CASE
}

// Adjoint of the velocity OE map (eq. magnetic-oe-map) with the damping
// factors D_l and the rho-weighted projector Psi frozen.  Per element and
// component, with W_q = Jdet w_q rho_q and shells l of the modal basis:
//   c = Psi^T W u*,  w_l = Psi_l c_l,  u' = sum_l D_l w_l,
//   e' = e + sum_{l >= 1} (1 - D_l^2)/2 sum_d w_{l,d}^2.
// For adjoints (lam_u', lam_e'): mu_l = D_l lam_u' + [l >= 1](1 - D_l^2) w_l lam_e',
// lam_c[alpha] = sum_q Psi[q][alpha] mu_{l(alpha)}[q], lam_u = W Psi lam_c, and
// lam_e = lam_e'.  lam holds (e, u) and is updated in place (u part).
template <int P>
__global__ void __launch_bounds__(OCfg<P>::threads) k_adj_vel_oe(const double* __restrict__ rho,
                                                                 double* __restrict__ lam,
                                                                 const double* __restrict__ ustar,
                                                                 const double* __restrict__ Psi,
                                                                 const double* __restrict__ frzD,
                                                                 const Tab* __restrict__ T, Mesh M) {
  using C = OCfg<P>;
  constexpr int n = C::n, n2 = C::n2, EB = C::EB, SW = C::SW;
  __shared__ double sPsi[EB][n2 * n2];
  __shared__ double sWu[3][EB * SW];
  __shared__ double sc[3][EB * SW];
  __shared__ double smu[3][n][EB * SW];
  const size_t N = (size_t)M.K * n2;
  const int tid = threadIdx.x, el = tid / SW, q = tid % SW;
  const bool node = q < n2;
  const int k = blockIdx.x * EB + el;
  const bool valid = k < M.K && node;
  const int kk = k < M.K ? k : M.K - 1;
  const int qq = node ? q : 0;
  const int i = qq % n, j = qq / n;
  for (int t = q; t < n2 * n2; t += SW) sPsi[el][t] = Psi[(size_t)kk * n2 * n2 + t];
  const size_t gq = (size_t)kk * n2 + qq;
  const double W = node ? M.Jdet * T->wp[i] * T->wp[j] * rho[gq] : 0.0;
  double lu[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sWu[d][tid] = node ? W * ustar[d * N + gq] : 0.0;
    lu[d] = node ? lam[(1 + d) * N + gq] : 0.0;
  }
  const double le = node ? lam[gq] : 0.0;
  double D[n];
#pragma unroll
  for (int l = 0; l < n; ++l) D[l] = frzD[(size_t)kk * n + l];
  __syncthreads();
  if (node) {  // c_alpha (lane q plays alpha)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
#pragma unroll
      for (int t = 0; t < n2; ++t) s = fma(sPsi[el][t * n2 + q], sWu[d][el * SW + t], s);
      sc[d][tid] = s;
    }
  }
  __syncthreads();
  if (node) {  // mu_l at node q
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int l = 0; l <= P; ++l) {
        double wl = 0.0;
#pragma unroll
        for (int al = l * l; al < (l + 1) * (l + 1); ++al) wl = fma(sc[d][el * SW + al], sPsi[el][q * n2 + al], wl);
        double mu = D[l] * lu[d];
        if (l > 0) mu = fma(fma(-D[l], D[l], 1.0) * wl, le, mu);
        smu[d][l][tid] = mu;
      }
    }
  }
  __syncthreads();
  if (node) {  // lam_c[alpha] (lane q plays alpha, in shell l)
    int l = 0;
#pragma unroll
    for (int ll = 1; ll <= P; ++ll)
      if (q >= ll * ll) l = ll;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
#pragma unroll
      for (int t = 0; t < n2; ++t) s = fma(sPsi[el][t * n2 + q], smu[d][l][el * SW + t], s);
      sc[d][tid] = s;
    }
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
#pragma unroll
      for (int al = 0; al < n2; ++al) s = fma(sPsi[el][q * n2 + al], sc[d][el * SW + al], s);
      lam[(1 + d) * N + gq] = W * s;
    }
  }
}

void stab_vel_adjoint(int p, const double* rho, double* lam, const double* ustar, const double* chol,
                      const double* frzD, const Tab* T, const Mesh& M, cudaStream_t st) {
#define MHD_ADJ_VOE(PP)                                                                                    \
  k_adj_vel_oe<PP><<<(unsigned)((M.K + OCfg<PP>::EB - 1) / OCfg<PP>::EB), OCfg<PP>::threads, 0, st>>>( \
      rho, lam, ustar, chol, frzD, T, M)
  switch (p) {
    case 1: MHD_ADJ_VOE(1); break;
    case 2: MHD_ADJ_VOE(2); break;
    case 3: MHD_ADJ_VOE(3); break;
    case 4: MHD_ADJ_VOE(4); break;
  }
#undef MHD_ADJ_VOE
}

MHD_OOB_READER(oob_stab)

}  // namespace mhd
