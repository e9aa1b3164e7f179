// Magnetic-velocity stage kernels (§3.3, eq. magnetic-dae, Algorithm 2).
//
// One SSP stage of the magnetic substep is three element kernels:
//   k_mag_J   element loads of the weak curl (eq. mag-current-proj):
//             (J, chi)_A = (B, curl chi)_B with the exact magnetic product
//             (Gauss(k+2) on R_h^k, Gauss(k+1) on V_h^k; eq.
//             magnetic-inner-product), sum-factorised through the exact
//             GLL(k+1) mass matrix.  Written closure-sized per element.
//   k_mag_E   assembles J_h over shared DOFs (lumped A-product, eq.
//             aux-inner-product: pointwise division), evaluates u_h and B_h at
//             the auxiliary nodes, writes the lumped Ohm-law loads of E_h
//             (eq. mag-electric-proj; element-wise quadrature at shared nodes),
//             forms the Lorentz load as the algebraic transpose of C_h
//             (eq. semi-vel), the Ohmic heating (eq. ohmic-heating), and the
//             SSP combination of (u, e).
//   k_mag_B   assembles E_h and applies the strong discrete curl
//             dB/dt = -curl E_h on the DOFs each element owns, then the SSP
//             combination of B (divergence-free by construction, Theorem
//             magnetic-divergence).
// Shared DOFs are assembled by every element that needs them in one canonical
// order (south-west contribution first), so all copies agree bitwise.
#include "mhd_internal.cuh"

namespace mhd {

template <int P, int KM>
struct MD {
  static constexpr int n = P + 1, n2 = n * n, mm = KM + 1, mL = KM + 2;
  static constexpr int NX = mm * mL;   // N_x family / Y-type arrays: a < mm (Gauss x), b < mL (GLL y)
  static constexpr int NY = mL * mm;   // N_y family / X-type arrays: a < mL (GLL x), b < mm (Gauss y)
  static constexpr int NW = mL * mL;   // W family
  static constexpr int NZ = mm * mm;   // owned DOFs / B_z
  static constexpr int EB = 16;        // elements per block
  static constexpr int TH = 256;       // threads per block
};

// ---- assembly of closure values from element loads ----------------------------
// W-type closure node (a, b), a, b < mL, of element (ex, ey).
template <int P, int KM>
__device__ __forceinline__ double assemble_W(const double* __restrict__ Lz, int ex, int ey, int a, int b,
                                             const Mesh& M, double iJ, const Tab* T) {
  using D = MD<P, KM>;
  int ox = ex, oy = ey, ao = a, bo = b;
  if (a == D::mL - 1) { ox = wrap(ex + 1, M.nx); ao = 0; }
  if (b == D::mL - 1) { oy = wrap(ey + 1, M.ny); bo = 0; }
  const int wx = wrap(ox - 1, M.nx), sy = wrap(oy - 1, M.ny);
  double v = 0.0;
  if (ao == 0 && bo == 0) v += Lz[(size_t)(sy * M.nx + wx) * D::NW + (D::mL - 1) * D::mL + (D::mL - 1)];
  if (bo == 0) v += Lz[(size_t)(sy * M.nx + ox) * D::NW + (D::mL - 1) * D::mL + ao];
  if (ao == 0) v += Lz[(size_t)(oy * M.nx + wx) * D::NW + bo * D::mL + (D::mL - 1)];
  v += Lz[(size_t)(oy * M.nx + ox) * D::NW + bo * D::mL + ao];
  double wa = ao == 0 ? 2.0 * T->wL[0] : T->wL[ao];
  double wb = bo == 0 ? 2.0 * T->wL[0] : T->wL[bo];
  return v / (wa * wb) * iJ;
}

// Y-type (N_x) closure node (a < mm, b < mL).
template <int P, int KM>
__device__ __forceinline__ double assemble_Nx(const double* __restrict__ Lx, int ex, int ey, int a, int b,
                                              const Mesh& M, double iJ, const Tab* T) {
  using D = MD<P, KM>;
  int oy = ey, bo = b;
  if (b == D::mL - 1) { oy = wrap(ey + 1, M.ny); bo = 0; }
  const int sy = wrap(oy - 1, M.ny);
  double v = 0.0;
  if (bo == 0) v += Lx[(size_t)(sy * M.nx + ex) * D::NX + (D::mL - 1) * D::mm + a];
  v += Lx[(size_t)(oy * M.nx + ex) * D::NX + bo * D::mm + a];
  double wb = bo == 0 ? 2.0 * T->wL[0] : T->wL[bo];
  return v / (T->wG[a] * wb) * iJ;
}

// X-type (N_y) closure node (a < mL, b < mm).
template <int P, int KM>
__device__ __forceinline__ double assemble_Ny(const double* __restrict__ Ly, int ex, int ey, int a, int b,
                                              const Mesh& M, double iJ, const Tab* T) {
  using D = MD<P, KM>;
  int ox = ex, ao = a;
  if (a == D::mL - 1) { ox = wrap(ex + 1, M.nx); ao = 0; }
  const int wx = wrap(ox - 1, M.nx);
  double v = 0.0;
  if (ao == 0) v += Ly[(size_t)(ey * M.nx + wx) * D::NY + b * D::mL + (D::mL - 1)];
  v += Ly[(size_t)(ey * M.nx + ox) * D::NY + b * D::mL + ao];
  double wa = ao == 0 ? 2.0 * T->wL[0] : T->wL[ao];
  return v / (wa * T->wG[b]) * iJ;
}

// B closure loads: Bx (X-type, [b < mm][a < mL]) and By (Y-type, [b < mL][a < mm]).
template <int P, int KM>
__device__ __forceinline__ double closure_Bx(const double* __restrict__ Bx, int ex, int ey, int a, int b,
                                             const Mesh& M) {
  using D = MD<P, KM>;
  if (a == D::mL - 1) return Bx[(size_t)(ey * M.nx + wrap(ex + 1, M.nx)) * D::NZ + b * D::mm];
  return Bx[(size_t)(ey * M.nx + ex) * D::NZ + b * D::mm + a];
}
template <int P, int KM>
__device__ __forceinline__ double closure_By(const double* __restrict__ By, int ex, int ey, int a, int b,
                                             const Mesh& M) {
  using D = MD<P, KM>;
  if (b == D::mL - 1) return By[(size_t)(wrap(ey + 1, M.ny) * M.nx + ex) * D::NZ + a];
  return By[(size_t)(ey * M.nx + ex) * D::NZ + b * D::mm + a];
}

#define FLAT_LOOP(ITEMS) for (int idx = threadIdx.x; idx < D::EB * (ITEMS); idx += blockDim.x)

// ============================ k_mag_J ==========================================
template <int P, int KM>
struct SJ {
  using D = MD<P, KM>;
  double bx[D::NY], by[D::NX], bz[D::NZ];
  double t1[D::mm * D::mL];   // [j < mm][a < mL]  sum_i Bx[j][i] ML[i][a]
  double t2[D::mL * D::mm];   // [b < mL][i < mm]  sum_j ML[j][b] By[j][i]
  double ta[D::NZ];           // Bz rows to Gauss x
  double bzg[D::NZ];          // Bz at Gauss(k)^2: [d][a]
};

template <int P, int KM>
__global__ void __launch_bounds__(256) k_mag_J(const double* __restrict__ Bx, const double* __restrict__ By,
                                               const double* __restrict__ Bz, double* __restrict__ LJx,
                                               double* __restrict__ LJy, double* __restrict__ LJz,
                                               const Tab* __restrict__ T, Mesh M) {
  using D = MD<P, KM>;
  extern __shared__ double smem_raw[];
  SJ<P, KM>* S = reinterpret_cast<SJ<P, KM>*>(smem_raw);
  const int k0 = blockIdx.x * D::EB;
  // stage 1: closures
  constexpr int I1 = D::NY + D::NX + D::NZ;
  FLAT_LOOP(I1) {
    int e = idx / I1, it = idx % I1, k = min(k0 + e, M.K - 1);
    int ex = k % M.nx, ey = k / M.nx;
    if (it < D::NY) { int a = it % D::mL, b = it / D::mL; S[e].bx[it] = closure_Bx<P, KM>(Bx, ex, ey, a, b, M); }
    else if (it < D::NY + D::NX) { it -= D::NY; int a = it % D::mm, b = it / D::mm; S[e].by[it] = closure_By<P, KM>(By, ex, ey, a, b, M); }
    else { it -= D::NY + D::NX; S[e].bz[it] = Bz[(size_t)k * D::NZ + it]; }
  }
  __syncthreads();
  // stage 2: t1, t2 (mass contractions) and the x-pass of Bz to Gauss points
  constexpr int I2 = D::mm * D::mL + D::mL * D::mm + D::NZ;
  FLAT_LOOP(I2) {
    int e = idx / I2, it = idx % I2;
    if (it < D::mm * D::mL) {
      int j = it / D::mL, a = it % D::mL;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < D::mL; ++i) s = fma(S[e].bx[j * D::mL + i], T->ML[i][a], s);
      S[e].t1[it] = s;
    } else if (it < 2 * D::mm * D::mL) {
      it -= D::mm * D::mL;
      int b = it / D::mm, i = it % D::mm;
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < D::mL; ++j) s = fma(T->ML[j][b], S[e].by[j * D::mm + i], s);
      S[e].t2[it] = s;
    } else {
      it -= 2 * D::mm * D::mL;
      int r = it / D::mm, a = it % D::mm;  // Bz row r (GLL(k) y), Gauss x point a
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) s = fma(T->M_G[a][c], S[e].bz[r * D::mm + c], s);
      S[e].ta[it] = s;
    }
  }
  __syncthreads();
  // stage 3: W loads and the y-pass of Bz
  const double cy = 2.0 / M.hy * M.Jdet, cx = 2.0 / M.hx * M.Jdet;
  constexpr int I3 = D::NW + D::NZ;
  FLAT_LOOP(I3) {
    int e = idx / I3, it = idx % I3, k = k0 + e;
    if (it < D::NW) {
      int b = it / D::mL, a = it % D::mL;
      double z1 = 0.0, z2 = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) {
        z1 = fma(T->wG[j] * T->dL_G[j][b], S[e].t1[j * D::mL + a], z1);
        z2 = fma(T->wG[j] * T->dL_G[j][a], S[e].t2[b * D::mm + j], z2);
      }
      if (k < M.K) LJz[(size_t)k * D::NW + it] = fma(cy, z1, -cx * z2);
    } else {
      it -= D::NW;
      int d = it / D::mm, a = it % D::mm;
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < D::mm; ++r) s = fma(T->M_G[d][r], S[e].ta[r * D::mm + a], s);
      S[e].bzg[it] = s;
    }
  }
  __syncthreads();
  // stage 4: N loads
  constexpr int I4 = D::NX + D::NY;
  FLAT_LOOP(I4) {
    int e = idx / I4, it = idx % I4, k = k0 + e;
    if (k >= M.K) continue;
    if (it < D::NX) {  // J_x: a < mm (Gauss x), b < mL
      int b = it / D::mm, a = it % D::mm;
      double s = 0.0;
#pragma unroll
      for (int d = 0; d < D::mm; ++d) s = fma(T->wG[d] * T->dL_G[d][b], S[e].bzg[d * D::mm + a], s);
      LJx[(size_t)k * D::NX + it] = -cy * T->wG[a] * s;
    } else {  // J_y: a < mL (GLL x), b < mm
      it -= D::NX;
      int b = it / D::mL, a = it % D::mL;
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) s = fma(T->wG[c] * T->dL_G[c][a], S[e].bzg[b * D::mm + c], s);
      LJy[(size_t)k * D::NY + it] = cx * T->wG[b] * s;
    }
  }
}

// ============================ k_mag_E ==========================================
template <int P, int KM>
struct SE {
  using D = MD<P, KM>;
  double jx[D::NX], jy[D::NY], jz[D::NW];
  double bx[D::NY], by[D::NX], bz[D::NZ];
  double u[3][D::n2], rho[D::n2];
  double ug[2][D::n * D::mm];    // u_y, u_z rows to Gauss x: [j][a]
  double ul[3][D::n * D::mL];    // u_x, u_y, u_z rows to GLL(k+1) x
  double bxg[D::NZ];             // Bx rows (Gauss y) to Gauss x
  double byl[D::NW];             // By rows (GLL y) to GLL x  (= By at W nodes)
  double bzg[D::NZ];             // Bz rows to Gauss x
  double bzl[D::mm * D::mL];     // Bz rows to GLL(k+1) x
  double unx[2][D::NX], uny[2][D::NY], uw[2][D::NW];
  double bxnx[D::NX], bznx[D::NX], byny[D::NY], bzny[D::NY], bxw[D::NW], bzw[D::NW];
  double ay_nx[D::NX], az_nx[D::NX], ax_ny[D::NY], az_ny[D::NY], ax_w[D::NW], ay_w[D::NW];
  double vx[D::n * D::mL], vy1[D::n * D::mm], vy2[D::n * D::mL], vz1[D::n * D::mm], vz2[D::n * D::mL];
  double jq[3][D::n2];           // J_h at the DG nodes (resistive part)
  double tq[3][D::n * D::mL];    // x-pass scratch of the resistive part
  double eta;
};

// mode 0: write du, de (residual test hook); mode 1: SSP combination into (uo, eo).
template <int P, int KM, int MODE>
__global__ void __launch_bounds__(256) k_mag_E(
    const double* __restrict__ LJx, const double* __restrict__ LJy, const double* __restrict__ LJz,
    const double* __restrict__ Bx, const double* __restrict__ By, const double* __restrict__ Bz,
    const double* __restrict__ u, const double* __restrict__ e, const double* __restrict__ rho,
    const double* __restrict__ eta, const double* __restrict__ u0, const double* __restrict__ e0,
    double* __restrict__ uo, double* __restrict__ eo, double* __restrict__ LEx, double* __restrict__ LEy,
    double* __restrict__ LEz, const Tab* __restrict__ T, Mesh M, const double* __restrict__ dtp, double dtfac,
    double ca, double cb, int first, int resistive) {
  using D = MD<P, KM>;
  extern __shared__ double smem_raw[];
  SE<P, KM>* S = reinterpret_cast<SE<P, KM>*>(smem_raw);
  const int k0 = blockIdx.x * D::EB;
  const size_t N = (size_t)M.K * D::n2;
  const double iJ = 1.0 / M.Jdet;
  // stage 1: J closure (assembled), B closure, u, rho, eta
  constexpr int I1 = D::NX + D::NY + D::NW + D::NY + D::NX + D::NZ + 4 * D::n2 + 1;
  FLAT_LOOP(I1) {
    int el = idx / I1, it = idx % I1, k = min(k0 + el, M.K - 1);
    int ex = k % M.nx, ey = k / M.nx;
    if (it < D::NX) { S[el].jx[it] = assemble_Nx<P, KM>(LJx, ex, ey, it % D::mm, it / D::mm, M, iJ, T); continue; }
    it -= D::NX;
    if (it < D::NY) { S[el].jy[it] = assemble_Ny<P, KM>(LJy, ex, ey, it % D::mL, it / D::mL, M, iJ, T); continue; }
    it -= D::NY;
    if (it < D::NW) { S[el].jz[it] = assemble_W<P, KM>(LJz, ex, ey, it % D::mL, it / D::mL, M, iJ, T); continue; }
    it -= D::NW;
    if (it < D::NY) { S[el].bx[it] = closure_Bx<P, KM>(Bx, ex, ey, it % D::mL, it / D::mL, M); continue; }
    it -= D::NY;
    if (it < D::NX) { S[el].by[it] = closure_By<P, KM>(By, ex, ey, it % D::mm, it / D::mm, M); continue; }
    it -= D::NX;
    if (it < D::NZ) { S[el].bz[it] = Bz[(size_t)k * D::NZ + it]; continue; }
    it -= D::NZ;
    if (it < 3 * D::n2) { int d = it / D::n2, q = it % D::n2; S[el].u[d][q] = u[d * N + (size_t)k * D::n2 + q]; continue; }
    it -= 3 * D::n2;
    if (it < D::n2) { S[el].rho[it] = rho[(size_t)k * D::n2 + it]; continue; }
    S[el].eta = resistive ? eta[k] : 0.0;
  }
  __syncthreads();
  // stage 2: x-passes
  constexpr int NUG = 2 * D::n * D::mm, NUL = 3 * D::n * D::mL;
  constexpr int I2 = NUG + NUL + D::NZ + D::NW + D::NZ + D::mm * D::mL;
  FLAT_LOOP(I2) {
    int el = idx / I2, it = idx % I2;
    auto& s = S[el];
    if (it < NUG) {  // u_y, u_z to Gauss x
      int d = it / (D::n * D::mm), r = it % (D::n * D::mm), j = r / D::mm, a = r % D::mm;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D::n; ++i) v = fma(T->P_G[a][i], s.u[1 + d][j * D::n + i], v);
      s.ug[d][r] = v;
      continue;
    }
    it -= NUG;
    if (it < NUL) {  // u_x, u_y, u_z to GLL(k+1) x
      int d = it / (D::n * D::mL), r = it % (D::n * D::mL), j = r / D::mL, a = r % D::mL;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D::n; ++i) v = fma(T->P_L[a][i], s.u[d][j * D::n + i], v);
      s.ul[d][r] = v;
      continue;
    }
    it -= NUL;
    if (it < D::NZ) {  // Bx rows (Gauss y) to Gauss x
      int j = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D::mL; ++i) v = fma(T->L_G[a][i], s.bx[j * D::mL + i], v);
      s.bxg[it] = v;
      continue;
    }
    it -= D::NZ;
    if (it < D::NW) {  // By rows (GLL y) to GLL x
      int j = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D::mm; ++i) v = fma(T->G_L[a][i], s.by[j * D::mm + i], v);
      s.byl[it] = v;
      continue;
    }
    it -= D::NW;
    if (it < D::NZ) {  // Bz rows to Gauss x
      int j = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D::mm; ++i) v = fma(T->M_G[a][i], s.bz[j * D::mm + i], v);
      s.bzg[it] = v;
      continue;
    }
    it -= D::NZ;
    {  // Bz rows to GLL(k+1) x
      int j = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D::mm; ++i) v = fma(T->M_L[a][i], s.bz[j * D::mm + i], v);
      s.bzl[it] = v;
    }
  }
  __syncthreads();
  // stage 3: y-passes to the auxiliary families
  constexpr int I3 = 2 * D::NX + 2 * D::NY + 2 * D::NW + D::NX + D::NX + D::NY + D::NY + D::NW + D::NW;
  FLAT_LOOP(I3) {
    int el = idx / I3, it = idx % I3;
    auto& s = S[el];
    if (it < 2 * D::NX) {  // u_y, u_z at N_x: GLL(k+1) y from GLL(p)
      int d = it / D::NX, r = it % D::NX, b = r / D::mm, a = r % D::mm;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::n; ++j) v = fma(T->P_L[b][j], s.ug[d][j * D::mm + a], v);
      s.unx[d][r] = v;
      continue;
    }
    it -= 2 * D::NX;
    if (it < 2 * D::NY) {  // u_x, u_z at N_y: Gauss y
      int d = it / D::NY, r = it % D::NY, b = r / D::mL, a = r % D::mL;
      const double* src = d == 0 ? s.ul[0] : s.ul[2];
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::n; ++j) v = fma(T->P_G[b][j], src[j * D::mL + a], v);
      s.uny[d][r] = v;
      continue;
    }
    it -= 2 * D::NY;
    if (it < 2 * D::NW) {  // u_x, u_y at W
      int d = it / D::NW, r = it % D::NW, b = r / D::mL, a = r % D::mL;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::n; ++j) v = fma(T->P_L[b][j], s.ul[d][j * D::mL + a], v);
      s.uw[d][r] = v;
      continue;
    }
    it -= 2 * D::NW;
    if (it < D::NX) {  // Bx at N_x: Gauss y -> GLL y
      int b = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) v = fma(T->G_L[b][j], s.bxg[j * D::mm + a], v);
      s.bxnx[it] = v;
      continue;
    }
    it -= D::NX;
    if (it < D::NX) {  // Bz at N_x: GLL(k) y -> GLL(k+1) y
      int b = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) v = fma(T->M_L[b][j], s.bzg[j * D::mm + a], v);
      s.bznx[it] = v;
      continue;
    }
    it -= D::NX;
    if (it < D::NY) {  // By at N_y: GLL y -> Gauss y
      int b = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::mL; ++j) v = fma(T->L_G[b][j], s.byl[j * D::mL + a], v);
      s.byny[it] = v;
      continue;
    }
    it -= D::NY;
    if (it < D::NY) {  // Bz at N_y: GLL(k) y -> Gauss y
      int b = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) v = fma(T->M_G[b][j], s.bzl[j * D::mL + a], v);
      s.bzny[it] = v;
      continue;
    }
    it -= D::NY;
    if (it < D::NW) {  // Bx at W: Gauss y -> GLL y
      int b = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) v = fma(T->G_L[b][j], s.bx[j * D::mL + a], v);
      s.bxw[it] = v;
      continue;
    }
    it -= D::NW;
    {  // Bz at W
      int b = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) v = fma(T->M_L[b][j], s.bzl[j * D::mL + a], v);
      s.bzw[it] = v;
    }
  }
  __syncthreads();
  // stage 4: pointwise E loads (lumped weights) and Lorentz products
  const double Jd = M.Jdet;
  constexpr int I4 = D::NX + D::NY + D::NW;
  FLAT_LOOP(I4) {
    int el = idx / I4, it = idx % I4, k = k0 + el;
    auto& s = S[el];
    if (it < D::NX) {
      int b = it / D::mm, a = it % D::mm;
      double w = Jd * T->wG[a] * T->wL[b];
      double by_ = s.by[it], bz_ = s.bznx[it], jx_ = s.jx[it];
      if (k < M.K) LEx[(size_t)k * D::NX + it] = w * fma(s.unx[1][it], by_, -s.unx[0][it] * bz_);
      s.ay_nx[it] = -w * bz_ * jx_;
      s.az_nx[it] = w * by_ * jx_;
    } else if (it < D::NX + D::NY) {
      it -= D::NX;
      int b = it / D::mL, a = it % D::mL;
      double w = Jd * T->wL[a] * T->wG[b];
      double bx_ = s.bx[it], bz_ = s.bzny[it], jy_ = s.jy[it];
      if (k < M.K) LEy[(size_t)k * D::NY + it] = w * fma(s.uny[0][it], bz_, -s.uny[1][it] * bx_);
      s.ax_ny[it] = w * bz_ * jy_;
      s.az_ny[it] = -w * bx_ * jy_;
    } else {
      it -= D::NX + D::NY;
      int b = it / D::mL, a = it % D::mL;
      double w = Jd * T->wL[a] * T->wL[b];
      double bx_ = s.bxw[it], by_ = s.byl[it], jz_ = s.jz[it];
      if (k < M.K) LEz[(size_t)k * D::NW + it] = w * fma(s.uw[1][it], bx_, -s.uw[0][it] * by_);
      s.ax_w[it] = -w * by_ * jz_;
      s.ay_w[it] = w * bx_ * jz_;
    }
  }
  __syncthreads();
  // stage 5: transposed y-pass onto the DG y-nodes
  constexpr int I5 = D::n * D::mL + D::n * D::mm + D::n * D::mL + D::n * D::mm + D::n * D::mL;
  FLAT_LOOP(I5) {
    int el = idx / I5, it = idx % I5;
    auto& s = S[el];
    if (it < D::n * D::mL) {
      int j = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D::mm; ++b) v = fma(T->P_G[b][j], s.ax_ny[b * D::mL + a], v);
#pragma unroll
      for (int b = 0; b < D::mL; ++b) v = fma(T->P_L[b][j], s.ax_w[b * D::mL + a], v);
      s.vx[it] = v;
      continue;
    }
    it -= D::n * D::mL;
    if (it < D::n * D::mm) {
      int j = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D::mL; ++b) v = fma(T->P_L[b][j], s.ay_nx[b * D::mm + a], v);
      s.vy1[it] = v;
      continue;
    }
    it -= D::n * D::mm;
    if (it < D::n * D::mL) {
      int j = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D::mL; ++b) v = fma(T->P_L[b][j], s.ay_w[b * D::mL + a], v);
      s.vy2[it] = v;
      continue;
    }
    it -= D::n * D::mL;
    if (it < D::n * D::mm) {
      int j = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D::mL; ++b) v = fma(T->P_L[b][j], s.az_nx[b * D::mm + a], v);
      s.vz1[it] = v;
      continue;
    }
    it -= D::n * D::mm;
    {
      int j = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D::mm; ++b) v = fma(T->P_G[b][j], s.az_ny[b * D::mL + a], v);
      s.vz2[it] = v;
    }
  }
  __syncthreads();
  // stage 5b (resistive only): J_h at the DG nodes, x-pass then y-pass
  bool any_res = false;
  if (resistive) {
    // x-pass: Jx rows (GLL y, b < mL) Gauss->DG x; Jy rows (Gauss y) GLL->DG x; Jz rows GLL->DG x
    constexpr int IR1 = D::mL * D::n + D::mm * D::n + D::mL * D::n;
    FLAT_LOOP(IR1) {
      int el = idx / IR1, it = idx % IR1;
      auto& s = S[el];
      if (s.eta == 0.0) continue;
      if (it < D::mL * D::n) {
        int b = it / D::n, i = it % D::n;
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < D::mm; ++a) v = fma(T->G_P[i][a], s.jx[b * D::mm + a], v);
        s.tq[0][it] = v;
      } else if (it < D::mL * D::n + D::mm * D::n) {
        it -= D::mL * D::n;
        int b = it / D::n, i = it % D::n;
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < D::mL; ++a) v = fma(T->L_P[i][a], s.jy[b * D::mL + a], v);
        s.tq[1][it] = v;
      } else {
        it -= D::mL * D::n + D::mm * D::n;
        int b = it / D::n, i = it % D::n;
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < D::mL; ++a) v = fma(T->L_P[i][a], s.jz[b * D::mL + a], v);
        s.tq[2][it] = v;
      }
    }
    __syncthreads();
    constexpr int IR2 = 3 * D::n2;
    FLAT_LOOP(IR2) {
      int el = idx / IR2, it = idx % IR2;
      auto& s = S[el];
      if (s.eta == 0.0) continue;
      int d = it / D::n2, q = it % D::n2, j = q / D::n, i = q % D::n;
      double v = 0.0;
      if (d == 0) {
#pragma unroll
        for (int b = 0; b < D::mL; ++b) v = fma(T->L_P[j][b], s.tq[0][b * D::n + i], v);
      } else if (d == 1) {
#pragma unroll
        for (int b = 0; b < D::mm; ++b) v = fma(T->G_P[j][b], s.tq[1][b * D::n + i], v);
      } else {
#pragma unroll
        for (int b = 0; b < D::mL; ++b) v = fma(T->L_P[j][b], s.tq[2][b * D::n + i], v);
      }
      s.jq[d][q] = v;
    }
    __syncthreads();
    // resistive loads R_n = eta sum_q Jdet w_q J(x_q) phi_n(x_q), added to the E loads
    // (each element adds only to its own closure loads)
    constexpr int IR3 = D::NX + D::NY + D::NW;
    FLAT_LOOP(IR3) {
      int el = idx / IR3, it = idx % IR3, k = k0 + el;
      auto& s = S[el];
      if (s.eta == 0.0 || k >= M.K) continue;
      double r = 0.0;
      if (it < D::NX) {
        int b = it / D::mm, a = it % D::mm;
        for (int j = 0; j < D::n; ++j) {
          double t = 0.0;
#pragma unroll
          for (int i = 0; i < D::n; ++i) t = fma(T->wp[i] * T->G_P[i][a], s.jq[0][j * D::n + i], t);
          r = fma(T->wp[j] * T->L_P[j][b], t, r);
        }
        LEx[(size_t)k * D::NX + it] += s.eta * Jd * r;
      } else if (it < D::NX + D::NY) {
        it -= D::NX;
        int b = it / D::mL, a = it % D::mL;
        for (int j = 0; j < D::n; ++j) {
          double t = 0.0;
#pragma unroll
          for (int i = 0; i < D::n; ++i) t = fma(T->wp[i] * T->L_P[i][a], s.jq[1][j * D::n + i], t);
          r = fma(T->wp[j] * T->G_P[j][b], t, r);
        }
        LEy[(size_t)k * D::NY + it] += s.eta * Jd * r;
      } else {
        it -= D::NX + D::NY;
        int b = it / D::mL, a = it % D::mL;
        for (int j = 0; j < D::n; ++j) {
          double t = 0.0;
#pragma unroll
          for (int i = 0; i < D::n; ++i) t = fma(T->wp[i] * T->L_P[i][a], s.jq[2][j * D::n + i], t);
          r = fma(T->wp[j] * T->L_P[j][b], t, r);
        }
        LEz[(size_t)k * D::NW + it] += s.eta * Jd * r;
      }
    }
    any_res = true;
  }
  // stage 6: x-pass onto DG nodes, velocity and energy rates, SSP combination
  const double tau = MODE ? dtp[0] * dtfac : 0.0;
  constexpr int I6 = D::n2;
  FLAT_LOOP(I6) {
    int el = idx / I6, q = idx % I6, k = k0 + el;
    if (k >= M.K) continue;
    auto& s = S[el];
    int j = q / D::n, i = q % D::n;
    double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
    for (int a = 0; a < D::mL; ++a) {
      sx = fma(T->P_L[a][i], s.vx[j * D::mL + a], sx);
      sy = fma(T->P_L[a][i], s.vy2[j * D::mL + a], sy);
      sz = fma(T->P_L[a][i], s.vz2[j * D::mL + a], sz);
    }
#pragma unroll
    for (int a = 0; a < D::mm; ++a) {
      sy = fma(T->P_G[a][i], s.vy1[j * D::mm + a], sy);
      sz = fma(T->P_G[a][i], s.vz1[j * D::mm + a], sz);
    }
    double r_ = s.rho[q];
    double im = rcp(r_ * Jd * T->wp[i] * T->wp[j]);
    double du[3] = {sx * im, sy * im, sz * im};
    double de = 0.0;
    if (any_res && s.eta != 0.0) {
      double jx = s.jq[0][q], jy = s.jq[1][q], jz = s.jq[2][q];
      de = s.eta * fma(jx, jx, fma(jy, jy, jz * jz)) * rcp(r_);
    }
    size_t gq = (size_t)k * D::n2 + q;
    if (MODE == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) uo[d * N + gq] = du[d];
      eo[gq] = de;
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double raw = fma(tau, du[d], s.u[d][q]);
        uo[d * N + gq] = first ? raw : fma(ca, u0[d * N + gq], cb * raw);
      }
      double raw = fma(tau, de, e[gq]);
      eo[gq] = first ? raw : fma(ca, e0[gq], cb * raw);
    }
  }
}

// ============================ k_mag_B ==========================================
template <int P, int KM>
struct SB {
  using D = MD<P, KM>;
  double ex[D::NX], ey[D::NY], ez[D::NW];
  double ty[D::mm * D::mm];   // d/dx of E_y rows at GLL(k) x: [b < mm][a < mm]
  double tx[D::mL * D::mm];   // E_x rows (GLL y) to GLL(k) x: [b < mL][a < mm]
};

// mode 0: write dB; mode 1: SSP combination into Bo.
template <int P, int KM, int MODE>
__global__ void __launch_bounds__(256) k_mag_B(
    const double* __restrict__ LEx, const double* __restrict__ LEy, const double* __restrict__ LEz,
    const double* __restrict__ B, const double* __restrict__ B0, double* __restrict__ Bo, const Tab* __restrict__ T,
    Mesh M, const double* __restrict__ dtp, double dtfac, double ca, double cb, int first) {
  using D = MD<P, KM>;
  extern __shared__ double smem_raw[];
  SB<P, KM>* S = reinterpret_cast<SB<P, KM>*>(smem_raw);
  const int k0 = blockIdx.x * D::EB;
  const double iJ = 1.0 / M.Jdet;
  const size_t Z = (size_t)M.K * D::NZ;
  constexpr int I1 = D::NX + D::NY + D::NW;
  FLAT_LOOP(I1) {
    int el = idx / I1, it = idx % I1, k = min(k0 + el, M.K - 1);
    int ex = k % M.nx, ey = k / M.nx;
    if (it < D::NX) S[el].ex[it] = assemble_Nx<P, KM>(LEx, ex, ey, it % D::mm, it / D::mm, M, iJ, T);
    else if (it < D::NX + D::NY) { it -= D::NX; S[el].ey[it] = assemble_Ny<P, KM>(LEy, ex, ey, it % D::mL, it / D::mL, M, iJ, T); }
    else { it -= D::NX + D::NY; S[el].ez[it] = assemble_W<P, KM>(LEz, ex, ey, it % D::mL, it / D::mL, M, iJ, T); }
  }
  __syncthreads();
  constexpr int I2 = D::NZ + D::mL * D::mm;
  FLAT_LOOP(I2) {
    int el = idx / I2, it = idx % I2;
    auto& s = S[el];
    if (it < D::NZ) {  // d/dx E_y at GLL(k) x, rows Gauss y
      int b = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mL; ++c) v = fma(T->dL_M[a][c], s.ey[b * D::mL + c], v);
      s.ty[it] = v;
    } else {
      it -= D::NZ;
      int b = it / D::mm, a = it % D::mm;  // E_x rows (GLL y) to GLL(k) x
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) v = fma(T->G_M[a][c], s.ex[b * D::mm + c], v);
      s.tx[it] = v;
    }
  }
  __syncthreads();
  const double tau = MODE ? dtp[0] * dtfac : 0.0;
  const double ax = 2.0 / M.hx, ay = 2.0 / M.hy;
  constexpr int I3 = 3 * D::NZ;
  FLAT_LOOP(I3) {
    int el = idx / I3, it = idx % I3, k = k0 + el;
    if (k >= M.K) continue;
    auto& s = S[el];
    int comp = it / D::NZ, r = it % D::NZ, b = r / D::mm, a = r % D::mm;
    double dB;
    if (comp == 0) {  // Bx at (xL_a, zG_b): -d_y E_z
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mL; ++c) v = fma(T->dL_G[b][c], s.ez[c * D::mL + a], v);
      dB = -ay * v;
    } else if (comp == 1) {  // By at (zG_a, xL_b): d_x E_z
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mL; ++c) v = fma(T->dL_G[a][c], s.ez[b * D::mL + c], v);
      dB = ax * v;
    } else {  // Bz at (xM_a, xM_b): -(d_x E_y - d_y E_x)
      double vy = 0.0, vx = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) vy = fma(T->G_M[b][c], s.ty[c * D::mm + a], vy);
#pragma unroll
      for (int c = 0; c < D::mL; ++c) vx = fma(T->dL_M[b][c], s.tx[c * D::mm + a], vx);
      dB = -fma(ax, vy, -ay * vx);
    }
    size_t gi = comp * Z + (size_t)k * D::NZ + r;
    if (MODE == 0) Bo[gi] = dB;
    else {
      double raw = fma(tau, dB, B[gi]);
      Bo[gi] = first ? raw : fma(ca, B0[gi], cb * raw);
    }
  }
}

// ---- launchers ------------------------------------------------------------------
template <int P, int KM>
static void set_smem(const void* f, size_t bytes) {
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int P, int KM>
void mag_stage_impl(int mode, const double* B, const double* u, const double* e, const double* rho,
                    const double* eta, int resistive, const double* B0, const double* u0, const double* e0,
                    double* Bo, double* uo, double* eo, double* LJ, double* LE, const Tab* T, const Mesh& M,
                    const double* dtp, double dtfac, double ca, double cb, int first, cudaStream_t st) {
  using D = MD<P, KM>;
  const size_t Z = (size_t)M.K * D::NZ;
  double* LJx = LJ; double* LJy = LJ + (size_t)M.K * D::NX; double* LJz = LJy + (size_t)M.K * D::NY;
  double* LEx = LE; double* LEy = LE + (size_t)M.K * D::NX; double* LEz = LEy + (size_t)M.K * D::NY;
  unsigned blocks = (unsigned)((M.K + D::EB - 1) / D::EB);
  size_t sj = sizeof(SJ<P, KM>) * D::EB, se = sizeof(SE<P, KM>) * D::EB, sb = sizeof(SB<P, KM>) * D::EB;
  static bool init = false;
  if (!init) {
    set_smem<P, KM>((const void*)k_mag_J<P, KM>, sj);
    set_smem<P, KM>((const void*)k_mag_E<P, KM, 0>, se);
    set_smem<P, KM>((const void*)k_mag_E<P, KM, 1>, se);
    set_smem<P, KM>((const void*)k_mag_B<P, KM, 0>, sb);
    set_smem<P, KM>((const void*)k_mag_B<P, KM, 1>, sb);
    init = true;
  }
  k_mag_J<P, KM><<<blocks, D::TH, sj, st>>>(B, B + Z, B + 2 * Z, LJx, LJy, LJz, T, M);
  if (mode == 0) {
    k_mag_E<P, KM, 0><<<blocks, D::TH, se, st>>>(LJx, LJy, LJz, B, B + Z, B + 2 * Z, u, e, rho, eta, u0, e0, uo, eo,
                                                  LEx, LEy, LEz, T, M, dtp, dtfac, ca, cb, first, resistive);
    k_mag_B<P, KM, 0><<<blocks, D::TH, sb, st>>>(LEx, LEy, LEz, B, B0, Bo, T, M, dtp, dtfac, ca, cb, first);
  } else {
    k_mag_E<P, KM, 1><<<blocks, D::TH, se, st>>>(LJx, LJy, LJz, B, B + Z, B + 2 * Z, u, e, rho, eta, u0, e0, uo, eo,
                                                  LEx, LEy, LEz, T, M, dtp, dtfac, ca, cb, first, resistive);
    k_mag_B<P, KM, 1><<<blocks, D::TH, sb, st>>>(LEx, LEy, LEz, B, B0, Bo, T, M, dtp, dtfac, ca, cb, first);
  }
}

size_t mag_load_doubles(int p, int k, int K) {
  (void)p;
  int mm = k + 1, mL = k + 2;
  return (size_t)K * (2 * mm * mL + mL * mL);
}

void mag_stage(int p, int k, int mode, const double* B, const double* u, const double* e, const double* rho,
               const double* eta, int resistive, const double* B0, const double* u0, const double* e0, double* Bo,
               double* uo, double* eo, double* LJ, double* LE, const Tab* T, const Mesh& M, const double* dtp,
               double dtfac, double ca, double cb, int first, cudaStream_t st) {
#define MHD_MAG_CASE(PP, KK)                                                                                     \
  mag_stage_impl<PP, KK>(mode, B, u, e, rho, eta, resistive, B0, u0, e0, Bo, uo, eo, LJ, LE, T, M, dtp, dtfac, ca, \
                         cb, first, st)
  MHD_DISPATCH_PK(p, k, MHD_MAG_CASE);
#undef MHD_MAG_CASE
}

}  // namespace mhd
