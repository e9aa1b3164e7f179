// Pointwise and reduction kernels: host<->device layout permutation of the
// compatible fields, the nodal variable exchange (§3.4.1), the discretely
// divergence-free initial field from a potential, the CFL time step and the
// per-element diagnostic partials.
#include "mhd_internal.cuh"

namespace mhd {

// grid [NY][NX] (X = ex*mm + a, Y = ey*mm + b) <-> element-blocked [K][mm*mm].
__global__ void k_grid_to_blocked(const double* __restrict__ g, double* __restrict__ o, int nx, int ny, int mm) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)nx * ny * mm * mm;
  if (t >= tot) return;
  int NX = nx * mm;
  int X = (int)(t % NX), Y = (int)(t / NX);
  int ex = X / mm, a = X % mm, ey = Y / mm, b = Y % mm;
  o[((size_t)ey * nx + ex) * mm * mm + b * mm + a] = g[t];
}
__global__ void k_blocked_to_grid(const double* __restrict__ o, double* __restrict__ g, int nx, int ny, int mm) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)nx * ny * mm * mm;
  if (t >= tot) return;
  int NX = nx * mm;
  int X = (int)(t % NX), Y = (int)(t / NX);
  int ex = X / mm, a = X % mm, ey = Y / mm, b = Y % mm;
  g[t] = o[((size_t)ey * nx + ex) * mm * mm + b * mm + a];
}

void grid_to_blocked(const double* g, double* o, int nx, int ny, int mm, cudaStream_t st) {
  size_t tot = (size_t)nx * ny * mm * mm;
  k_grid_to_blocked<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(g, o, nx, ny, mm);
}
void blocked_to_grid(const double* o, double* g, int nx, int ny, int mm, cudaStream_t st) {
  size_t tot = (size_t)nx * ny * mm * mm;
  k_blocked_to_grid<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(o, g, nx, ny, mm);
}

// (rho, m, E_mech) -> (e, u) at every GLL node; Y = [e | u_x | u_y | u_z].
__global__ void k_cons_to_prim(const double* __restrict__ U, double* __restrict__ Y, size_t N) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  double rho = U[q], ir = rcp(rho);
  double ux = U[N + q] * ir, uy = U[2 * N + q] * ir, uz = U[3 * N + q] * ir;
  double ke = 0.5 * rho * fma(ux, ux, fma(uy, uy, uz * uz));
  Y[q] = (U[4 * N + q] - ke) * ir;
  Y[N + q] = ux; Y[2 * N + q] = uy; Y[3 * N + q] = uz;
}

// (e, u) -> (m, E_mech) with the frozen density.
__global__ void k_prim_to_cons(const double* __restrict__ Y, double* __restrict__ U, size_t N) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  double rho = U[q];
  double ux = Y[N + q], uy = Y[2 * N + q], uz = Y[3 * N + q];
  U[N + q] = rho * ux; U[2 * N + q] = rho * uy; U[3 * N + q] = rho * uz;
  U[4 * N + q] = fma(rho, Y[q], 0.5 * rho * fma(ux, ux, fma(uy, uy, uz * uz)));
}

// (rho, u, p) -> conservative.
__global__ void k_prim_in(const double* __restrict__ rho, const double* __restrict__ u, const double* __restrict__ p,
                          double* __restrict__ U, size_t N, double g) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  double r = rho[q], ux = u[q], uy = u[N + q], uz = u[2 * N + q];
  U[q] = r; U[N + q] = r * ux; U[2 * N + q] = r * uy; U[3 * N + q] = r * uz;
  U[4 * N + q] = p[q] / (g - 1.0) + 0.5 * r * (ux * ux + uy * uy + uz * uz);
}

// Vector-Jacobian product of k_prim_in at (rho, u): with lam = dJ/dU,
//   g_rho = lam_rho + u . lam_m + |u|^2/2 lam_E,
//   g_u   = rho lam_m + rho u lam_E,
//   g_p   = lam_E / (gamma - 1).
// G = [g_rho | g_u (3) | g_p], each [N].
__global__ void k_prim_in_vjp(const double* __restrict__ rho, const double* __restrict__ u,
                              const double* __restrict__ lam, double* __restrict__ G, size_t N, double ig1) {
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const double r = rho[q], ux = u[q], uy = u[N + q], uz = u[2 * N + q];
  const double lr = lam[q], lx = lam[N + q], ly = lam[2 * N + q], lz = lam[3 * N + q], le = lam[4 * N + q];
  const double u2 = fma(ux, ux, fma(uy, uy, uz * uz));
  G[q] = fma(0.5 * u2, le, fma(ux, lx, fma(uy, ly, fma(uz, lz, lr))));
  G[N + q] = r * fma(ux, le, lx);
  G[2 * N + q] = r * fma(uy, le, ly);
  G[3 * N + q] = r * fma(uz, le, lz);
  G[4 * N + q] = le * ig1;
}

void prim_in_vjp(const double* rho, const double* u, const double* lam, double* G, size_t N, double ig1,
                 cudaStream_t st) {
  k_prim_in_vjp<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rho, u, lam, G, N, ig1);
}

void cons_to_prim(const double* U, double* Y, size_t N, cudaStream_t st) {
  k_cons_to_prim<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(U, Y, N);
}
void prim_to_cons(const double* Y, double* U, size_t N, cudaStream_t st) {
  k_prim_to_cons<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(Y, U, N);
}
void prim_in(const double* rho, const double* u, const double* p, double* U, size_t N, double g, cudaStream_t st) {
  k_prim_in<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rho, u, p, U, N, g);
}

// B_par = B0 + grad^perp A_h on the owned R_h^k DOFs, A blocked [K][mm^2].
template <int KM>
__global__ void k_b_from_potential(const double* __restrict__ A, double Bx0, double By0, double* __restrict__ Bx,
                                   double* __restrict__ By, const Tab* __restrict__ T, Mesh M) {
  constexpr int mm = KM + 1, mL = KM + 2;
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)M.K * mm * mm) return;
  int k = (int)(t / (mm * mm)), r = (int)(t % (mm * mm)), b = r / mm, a = r % mm;
  int ex = k % M.nx, ey = k / M.nx;
  auto Acl = [&](int aa, int bb) {
    int ox = ex, oy = ey;
    if (aa == mL - 1) { ox = wrap(ex + 1, M.nx); aa = 0; }
    if (bb == mL - 1) { oy = wrap(ey + 1, M.ny); bb = 0; }
    return A[((size_t)oy * M.nx + ox) * mm * mm + bb * mm + aa];
  };
  double vx = 0.0, vy = 0.0;
  for (int c = 0; c < mL; ++c) {
    vx = fma(T->dL_G[b][c], Acl(a, c), vx);  // d/dy at (xL_a, zG_b)
    vy = fma(T->dL_G[a][c], Acl(c, b), vy);  // d/dx at (zG_a, xL_b)
  }
  Bx[t] = Bx0 - 2.0 / M.hy * vx;
  By[t] = By0 + 2.0 / M.hx * vy;
}

void b_from_potential(int k, const double* A, double Bx0, double By0, double* Bx, double* By, const Tab* T,
                      const Mesh& M, cudaStream_t st) {
  size_t tot = (size_t)M.K * (k + 1) * (k + 1);
  unsigned bl = (unsigned)((tot + 255) / 256);
  switch (k) {
    case 0: k_b_from_potential<0><<<bl, 256, 0, st>>>(A, Bx0, By0, Bx, By, T, M); break;
    case 1: k_b_from_potential<1><<<bl, 256, 0, st>>>(A, Bx0, By0, Bx, By, T, M); break;
    case 2: k_b_from_potential<2><<<bl, 256, 0, st>>>(A, Bx0, By0, Bx, By, T, M); break;
    case 3: k_b_from_potential<3><<<bl, 256, 0, st>>>(A, Bx0, By0, Bx, By, T, M); break;
    case 4: k_b_from_potential<4><<<bl, 256, 0, st>>>(A, Bx0, By0, Bx, By, T, M); break;
  }
}

// Element-wise L2 projection onto Q^k of data at the nq x nq Gauss points:
// C[b][a] = sum_{j,i} P[b][j] P[a][i] F[j][i], one thread per output node.
struct ProjTab {
  double P[MHD_NMAX * MHD_QMAX];
};

__global__ void k_l2_project(const double* __restrict__ fq, int nq, int mm, ProjTab T, double* __restrict__ out,
                             size_t K) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * mm * mm) return;
  size_t k = t / (mm * mm);
  int r = (int)(t % (mm * mm)), b = r / mm, a = r % mm;
  const double* F = fq + k * nq * nq;
  double c = 0.0;
  for (int j = 0; j < nq; ++j) {
    double row = 0.0;
    for (int i = 0; i < nq; ++i) row = fma(T.P[a * nq + i], F[j * nq + i], row);
    c = fma(T.P[b * nq + j], row, c);
  }
  out[t] = c;
}

void l2_project(int k, int nq, const double* fq, double* out, size_t K, cudaStream_t st) {
  ProjTab T;
  l2_projection_table(k, nq, T.P);
  size_t tot = K * (k + 1) * (k + 1);
  k_l2_project<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(fq, nq, k + 1, T, out, K);
}

// B_h of element k at its DG node (i, j) (tensor interpolation of the closures).
template <int P, int KM>
__device__ void B_at_dg(const double* __restrict__ B, size_t Z, const Tab* __restrict__ T, const Mesh& M, int k, int i,
                        int j, double out[3]) {
  constexpr int mm = KM + 1, mL = KM + 2;
  int ex = k % M.nx, ey = k / M.nx;
  const double* Bx = B;
  const double* By = B + Z;
  const double* Bz = B + 2 * Z;
  double bx = 0.0, by = 0.0, bz = 0.0;
  for (int b = 0; b < mm; ++b) {  // Bx: GLL(k+1) x (closure), Gauss y
    double row = 0.0;
    for (int a = 0; a < mL; ++a) {
      double v = a == mL - 1 ? Bx[((size_t)ey * M.nx + wrap(ex + 1, M.nx)) * mm * mm + b * mm]
                             : Bx[(size_t)k * mm * mm + b * mm + a];
      row = fma(T->L_P[i][a], v, row);
    }
    bx = fma(T->G_P[j][b], row, bx);
  }
  for (int b = 0; b < mL; ++b) {  // By: Gauss x, GLL(k+1) y (closure)
    double row = 0.0;
    for (int a = 0; a < mm; ++a) {
      double v = b == mL - 1 ? By[((size_t)wrap(ey + 1, M.ny) * M.nx + ex) * mm * mm + a]
                             : By[(size_t)k * mm * mm + b * mm + a];
      row = fma(T->G_P[i][a], v, row);
    }
    by = fma(T->L_P[j][b], row, by);
  }
  for (int b = 0; b < mm; ++b) {
    double row = 0.0;
    for (int a = 0; a < mm; ++a) row = fma(T->M_P[i][a], Bz[(size_t)k * mm * mm + b * mm + a], row);
    bz = fma(T->M_P[j][b], row, bz);
  }
  out[0] = bx; out[1] = by; out[2] = bz;
}

// Largest CFL rate (reading R2) over the DG nodes: atomicMax on the bits of a
// non-negative double.
template <int P, int KM>
__global__ void k_cfl(const double* __restrict__ U, const double* __restrict__ B, const Tab* __restrict__ T, Mesh M,
                      unsigned long long* __restrict__ maxbits) {
  constexpr int n = P + 1, n2 = n * n;
  size_t N = (size_t)M.K * n2, Z = (size_t)M.K * (KM + 1) * (KM + 1);
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double rate = 0.0;
  if (t < N) {
    int k = (int)(t / n2), q = (int)(t % n2);
    double Bv[3];
    B_at_dg<P, KM>(B, Z, T, M, k, q % n, q / n, Bv);
    double rho = U[t], ir = 1.0 / rho;
    double ux = U[N + t] * ir, uy = U[2 * N + t] * ir, uz = U[3 * N + t] * ir;
    double pr = (M.g - 1.0) * (U[4 * N + t] - 0.5 * rho * (ux * ux + uy * uy + uz * uz));
    double cf = sqrt((M.g * pr + Bv[0] * Bv[0] + Bv[1] * Bv[1] + Bv[2] * Bv[2]) * ir);
    rate = (2.0 * P + 1.0) * fmax((fabs(ux) + cf) / M.hx, (fabs(uy) + cf) / M.hy);
    if (!(rate >= 0.0)) rate = __longlong_as_double(0x7ff0000000000000ULL);  // non-finite -> +inf
  }
  unsigned long long bits = (unsigned long long)__double_as_longlong(rate);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, bits);
}

__global__ void k_finalize_dt(const unsigned long long* __restrict__ maxbits, double cfl, double* __restrict__ dt) {
  double r = __longlong_as_double((long long)*maxbits);
  dt[0] = cfl / r;
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// The reduced 2D2V stage needs m_z = 0 and B_z = 0 everywhere: flag any other
// value (NaN included) in the status word.  Every thread reaches the vote.
__global__ void k_check_planar(const double* __restrict__ mz, size_t N, const double* __restrict__ bz, size_t Z,
                               unsigned* __restrict__ status) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N + Z; i += (size_t)gridDim.x * blockDim.x) {
    const double v = i < N ? mz[i] : bz[i - N];
    bad |= !(v == 0.0);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NOT_PLANAR);
}

void check_planar(const double* mz, size_t N, const double* bz, size_t Z, unsigned* status, cudaStream_t st) {
  const size_t tot = N + Z;
  unsigned blocks = (unsigned)std::min<size_t>((tot + 255) / 256, 148 * 8);
  k_check_planar<<<blocks, 256, 0, st>>>(mz, N, bz, Z, status);
}

void cfl_dt(int p, int k, const double* U, const double* B, const Tab* T, const Mesh& M,
            unsigned long long* maxbits, double cfl, double* dt, cudaStream_t st) {
  cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), st);
  size_t N = (size_t)M.K * (p + 1) * (p + 1);
  unsigned bl = (unsigned)((N + 255) / 256);
#define MHD_CFL_CASE(PP, KK) k_cfl<PP, KK><<<bl, 256, 0, st>>>(U, B, T, M, maxbits)
  MHD_DISPATCH_PK(p, k, MHD_CFL_CASE);
#undef MHD_CFL_CASE
  k_finalize_dt<<<1, 1, 0, st>>>(maxbits, cfl, dt);
}

void set_scalar(double* ptr, double v, cudaStream_t st) { k_set_scalar<<<1, 1, 0, st>>>(ptr, v); }

// Per-element partials: [mass, mx, my, mz, E_kin, E_int, entropy, 2 E_mag,
// div metric, |B| max, rho min, p min] -> out[K][12].
template <int P, int KM>
__global__ void k_diag(const double* __restrict__ U, const double* __restrict__ B, const Tab* __restrict__ T, Mesh M,
                       double* __restrict__ out) {
  constexpr int n = P + 1, n2 = n * n, mm = KM + 1, mL = KM + 2;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M.K) return;
  size_t N = (size_t)M.K * n2, Z = (size_t)M.K * mm * mm;
  double acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1e300, 1e300};
  for (int q = 0; q < n2; ++q) {
    int i = q % n, j = q / n;
    double w = M.Jdet * T->wp[i] * T->wp[j];
    size_t t = (size_t)k * n2 + q;
    double rho = U[t], mx = U[N + t], my = U[2 * N + t], mz = U[3 * N + t], E = U[4 * N + t];
    double ke = 0.5 * (mx * mx + my * my + mz * mz) / rho;
    double pr = (M.g - 1.0) * (E - ke);
    acc[0] += w * rho; acc[1] += w * mx; acc[2] += w * my; acc[3] += w * mz;
    acc[4] += w * ke; acc[5] += w * pr / (M.g - 1.0);
    acc[6] += w * rho * (log(pr) - M.g * log(rho));
    double Bv[3];
    B_at_dg<P, KM>(B, Z, T, M, k, i, j, Bv);
    acc[9] = fmax(acc[9], sqrt(Bv[0] * Bv[0] + Bv[1] * Bv[1] + Bv[2] * Bv[2]));
    acc[10] = fmin(acc[10], rho);
    acc[11] = fmin(acc[11], pr);
  }
  // exact magnetic energy and the divergence metric
  int ex = k % M.nx, ey = k / M.nx;
  const double* Bx = B;
  const double* By = B + Z;
  const double* Bz = B + 2 * Z;
  double bx[mm][mL], by[mL][mm];
  for (int b = 0; b < mm; ++b)
    for (int a = 0; a < mL; ++a)
      bx[b][a] = a == mL - 1 ? Bx[MHD_CHK(((size_t)ey * M.nx + wrap(ex + 1, M.nx)) * mm * mm + b * mm, Z)]
                             : Bx[(size_t)k * mm * mm + b * mm + a];
  for (int b = 0; b < mL; ++b)
    for (int a = 0; a < mm; ++a)
      by[b][a] = b == mL - 1 ? By[MHD_CHK(((size_t)wrap(ey + 1, M.ny) * M.nx + ex) * mm * mm + a, Z)]
                             : By[(size_t)k * mm * mm + b * mm + a];
  double em = 0.0;
  for (int qy = 0; qy < mL; ++qy)
    for (int qx = 0; qx < mL; ++qx) {
      double vx = 0.0, vy = 0.0;
      for (int b = 0; b < mm; ++b)
        for (int a = 0; a < mL; ++a) vx += bx[b][a] * T->L_2[qx][a] * T->G_2[qy][b];
      for (int b = 0; b < mL; ++b)
        for (int a = 0; a < mm; ++a) vy += by[b][a] * T->G_2[qx][a] * T->L_2[qy][b];
      em += M.Jdet * T->w2[qx] * T->w2[qy] * (vx * vx + vy * vy);
    }
  for (int qy = 0; qy < mm; ++qy)
    for (int qx = 0; qx < mm; ++qx) {
      double vz = 0.0;
      for (int b = 0; b < mm; ++b)
        for (int a = 0; a < mm; ++a) vz += Bz[(size_t)k * mm * mm + b * mm + a] * T->M_G[qx][a] * T->M_G[qy][b];
      em += M.Jdet * T->wG[qx] * T->wG[qy] * vz * vz;
    }
  acc[7] = em;
  double dv = 0.0;
  for (int qy = 0; qy < mm; ++qy)
    for (int qx = 0; qx < mm; ++qx) {
      double dx = 0.0, dy = 0.0;
      for (int b = 0; b < mm; ++b)
        for (int a = 0; a < mL; ++a) dx += bx[b][a] * T->dL_G[qx][a] * (b == qy ? 1.0 : 0.0);
      for (int b = 0; b < mL; ++b)
        for (int a = 0; a < mm; ++a) dy += by[b][a] * (a == qx ? 1.0 : 0.0) * T->dL_G[qy][b];
      dv = fmax(dv, fabs(2.0 / M.hx * dx + 2.0 / M.hy * dy));
    }
  acc[8] = fmin(M.hx, M.hy) * dv;
  for (int c = 0; c < 12; ++c) out[(size_t)k * 12 + c] = acc[c];
}

void diag_partials(int p, int k, const double* U, const double* B, const Tab* T, const Mesh& M, double* out,
                   cudaStream_t st) {
  unsigned bl = (unsigned)((M.K + 127) / 128);
#define MHD_DIAG_CASE(PP, KK) k_diag<PP, KK><<<bl, 128, 0, st>>>(U, B, T, M, out)
  MHD_DISPATCH_PK(p, k, MHD_DIAG_CASE);
#undef MHD_DIAG_CASE
}

}  // namespace mhd

namespace mhd {
// FP64 FMA throughput probe: 8 independent dependency chains per thread, every
// lane active.  Used to report the measured FP64 issue peak next to the
// kernels' achieved rate.
__global__ void k_dfma_probe(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
}  // namespace mhd

extern "C" int mhd_fp64_peak(double* tflops) {
  if (!tflops) return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -3;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8, iters = 4096;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return -2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  mhd::k_dfma_probe<<<blocks, threads>>>(out, 64, 0.999, 1e-3);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    mhd::k_dfma_probe<<<blocks, threads>>>(out, iters, 0.999, 1e-3);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return -3;
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return 0;
}

// ---- test hook: the library's refined reciprocal on caller data ---------------
namespace mhd {
void set_error_message(const char* msg);
__global__ void k_rcp_check(const double* __restrict__ x, double* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = rcp(x[i]);
}
__global__ void k_sqrt_check(const double* __restrict__ x, double* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fsqrt(x[i]);
}
}  // namespace mhd

extern "C" int mhd_rcp_check(const double* x, double* y, long long n, void* stream) {
  if (!x || !y || n < 0) {
    mhd::set_error_message("null argument or negative length");
    return -1;
  }
  if (n == 0) return 0;
  const int th = 256;
  const long long blocks = (n + th - 1) / th;
  if (blocks > 0x7fffffffLL) {
    mhd::set_error_message("length too large for one launch");
    return -1;
  }
  mhd::k_rcp_check<<<(unsigned)blocks, th, 0, (cudaStream_t)stream>>>(x, y, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mhd::set_error_message(cudaGetErrorString(e));
    return -3;
  }
  return 0;
}

extern "C" int mhd_sqrt_check(const double* x, double* y, long long n, void* stream) {
  if (!x || !y || n < 0) {
    mhd::set_error_message("null argument or negative length");
    return -1;
  }
  if (n == 0) return 0;
  const int th = 256;
  const long long blocks = (n + th - 1) / th;
  if (blocks > 0x7fffffffLL) {
    mhd::set_error_message("length too large for one launch");
    return -1;
  }
  mhd::k_sqrt_check<<<(unsigned)blocks, th, 0, (cudaStream_t)stream>>>(x, y, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mhd::set_error_message(cudaGetErrorString(e));
    return -3;
  }
  return 0;
}

// ---- reflecting walls by the method of images ---------------------------------
// A walled domain [x0,x1] x [y0,y1] is stored as the periodic domain doubled in
// every walled direction; the physical elements are ex < pnx, ey < pny.  The
// image of a field is its reflection about x1 (and/or y1) with the parity of a
// mirror: the normal velocity is odd, the other fluid fields even; B has, per
// wall pair, the parity of a conducting wall (B_n odd, B_t even: B_n = 0 on the
// wall) or of a symmetry plane (B_n even, B_t odd).  Bit 0 of `walls` and
// `cond` is the x pair, bit 1 the y pair.  Every operator of the step is
// reflection-equivariant, so a mirror-symmetric state stays mirror-symmetric and
// its physical part is the solution with the walls (reading R24).
namespace mhd {

__device__ __forceinline__ int mirror_elem(int e, int pn, bool* refl) {
  *refl = e >= pn;
  return *refl ? 2 * pn - 1 - e : e;
}

template <int P>
__global__ void k_mirror_dg(double* __restrict__ U, Mesh M, int pnx, int pny, int walls) {
  constexpr int n = P + 1, n2 = n * n;
  const size_t N = (size_t)M.K * n2;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int k = (int)(t / n2), q = (int)(t % n2), i = q % n, j = q / n;
  const int ex = k % M.nx, ey = k / M.nx;
  bool rx = false, ry = false;
  const int sx = (walls & 1) ? mirror_elem(ex, pnx, &rx) : ex;
  const int sy = (walls & 2) ? mirror_elem(ey, pny, &ry) : ey;
  if (!rx && !ry) return;  // a physical node
  const int si = rx ? P - i : i, sj = ry ? P - j : j;
  const size_t s = MHD_CHK((size_t)(sy * M.nx + sx) * n2 + sj * n + si, N);
  U[t] = U[s];
  U[N + t] = rx ? -U[N + s] : U[N + s];
  U[2 * N + t] = ry ? -U[2 * N + s] : U[2 * N + s];
  U[3 * N + t] = U[3 * N + s];
  U[4 * N + t] = U[4 * N + s];
}

template <int KM>
__global__ void k_mirror_B(double* __restrict__ B, Mesh M, int pnx, int pny, int walls, int cond) {
  constexpr int mm = KM + 1;
  const size_t Z = (size_t)M.K * mm * mm;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * Z) return;
  const int comp = (int)(t / Z);
  const size_t o = t % Z;
  const int k = (int)(o / (mm * mm)), w = (int)(o % (mm * mm)), a = w % mm, b = w / mm;
  const int ex = k % M.nx, ey = k / M.nx;
  const int NX = M.nx * mm, NY = M.ny * mm, PX = pnx * mm, PY = pny * mm;
  const bool wx = walls & 1, wy = walls & 2, cx = cond & 1, cy = cond & 2;
  int c = ex * mm + a, r = ey * mm + b;  // global column / row of the DOF
  double sign = 1.0;
  bool plane_zero = false, image = false;
  if (comp == 0) {  // B_x: GLL(k+1) columns (mirror planes at c = 0, PX), Gauss rows
    if (wx && (c == 0 || c == PX)) plane_zero = cx;
    else if (wx && c > PX) { c = NX - c; image = true; sign *= cx ? -1.0 : 1.0; }
    if (wy && r >= PY) { r = NY - 1 - r; image = true; sign *= cy ? 1.0 : -1.0; }
  } else if (comp == 1) {  // B_y: Gauss columns, GLL(k+1) rows (mirror planes at r = 0, PY)
    if (wx && c >= PX) { c = NX - 1 - c; image = true; sign *= cx ? 1.0 : -1.0; }
    if (wy && (r == 0 || r == PY)) plane_zero = cy;
    else if (wy && r > PY) { r = NY - r; image = true; sign *= cy ? -1.0 : 1.0; }
  } else {  // B_z: GLL(k) nodes of the element, tangential to every wall
    if (wx && ex >= pnx) { c = (2 * pnx - 1 - ex) * mm + (KM - a); image = true; sign *= cx ? 1.0 : -1.0; }
    if (wy && ey >= pny) { r = (2 * pny - 1 - ey) * mm + (KM - b); image = true; sign *= cy ? 1.0 : -1.0; }
  }
  if (plane_zero) { B[t] = 0.0; return; }
  if (!image) return;
  // the source is a physical DOF off the mirror planes (no thread writes it)
  const int se = (r / mm) * M.nx + c / mm;
  B[t] = sign * B[MHD_CHK((size_t)comp * Z + (size_t)se * mm * mm + (r % mm) * mm + c % mm, 3 * Z)];
}

void mirror_fill(int p, int k, double* U, double* B, const Mesh& M, int pnx, int pny, int walls, int cond,
                 cudaStream_t st) {
  const size_t N = (size_t)M.K * (p + 1) * (p + 1), Z3 = 3 * (size_t)M.K * (k + 1) * (k + 1);
  const unsigned bN = (unsigned)((N + 255) / 256), bZ = (unsigned)((Z3 + 255) / 256);
  switch (p) {
    case 1: k_mirror_dg<1><<<bN, 256, 0, st>>>(U, M, pnx, pny, walls); break;
    case 2: k_mirror_dg<2><<<bN, 256, 0, st>>>(U, M, pnx, pny, walls); break;
    case 3: k_mirror_dg<3><<<bN, 256, 0, st>>>(U, M, pnx, pny, walls); break;
    case 4: k_mirror_dg<4><<<bN, 256, 0, st>>>(U, M, pnx, pny, walls); break;
  }
  switch (k) {
    case 0: k_mirror_B<0><<<bZ, 256, 0, st>>>(B, M, pnx, pny, walls, cond); break;
    case 1: k_mirror_B<1><<<bZ, 256, 0, st>>>(B, M, pnx, pny, walls, cond); break;
    case 2: k_mirror_B<2><<<bZ, 256, 0, st>>>(B, M, pnx, pny, walls, cond); break;
    case 3: k_mirror_B<3><<<bZ, 256, 0, st>>>(B, M, pnx, pny, walls, cond); break;
    case 4: k_mirror_B<4><<<bZ, 256, 0, st>>>(B, M, pnx, pny, walls, cond); break;
  }
}

MHD_OOB_READER(oob_misc)

}  // namespace mhd
