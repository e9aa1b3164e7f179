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
//
// Work mapping (the FP64 pipe is the bound: keep every lane busy, keep table
// reads uniform): a block holds EB = 16 elements; shared memory is laid out
// element-innermost ([quantity][item][element]) and a flat loop index is
// item * EB + element, so each half-warp evaluates one item for 16 elements.
// All lanes of a half-warp take the same branch and read the same table
// entries, which live in constant memory (broadcast reads).
#include <cstring>

#include "mhd_internal.cuh"

namespace mhd {

// The 1D tables the magnetic kernels read, in constant memory (broadcast
// reads), with the products of two table entries that their loops would
// otherwise form in every iteration rounded once on the host (the same
// IEEE product, so the results do not change).
struct MTab {
  double wp[MHD_NMAX], wL[MHD_LMAX], wG[MHD_NMAX];
  double ML[MHD_LMAX][MHD_LMAX];
  double dL_G[MHD_NMAX][MHD_LMAX], G_L[MHD_LMAX][MHD_NMAX], M_G[MHD_NMAX][MHD_NMAX], M_L[MHD_LMAX][MHD_NMAX];
  double P_G[MHD_NMAX][MHD_NMAX], P_L[MHD_LMAX][MHD_NMAX], dL_M[MHD_NMAX][MHD_LMAX], G_M[MHD_NMAX][MHD_NMAX];
  double L_P[MHD_NMAX][MHD_LMAX], G_P[MHD_NMAX][MHD_NMAX];
  double WG_P[MHD_NMAX][MHD_NMAX], WL_P[MHD_NMAX][MHD_LMAX];
  double iwLs[MHD_LMAX], iwG[MHD_NMAX];
  double wdL_G[MHD_NMAX][MHD_LMAX];  // wG_j dL_G[j][b]
  double W_GL[MHD_NMAX][MHD_LMAX];   // wG_a wL_b: lumped weight of an N_x node (a Gauss in x, b GLL in y)
  double W_LG[MHD_LMAX][MHD_NMAX];   // wL_a wG_b: N_y node
  double W_LL[MHD_LMAX][MHD_LMAX];   // wL_a wL_b: W node
  // reciprocal lumped weights of the three families, one product each
  double iW_LL[MHD_LMAX][MHD_LMAX];  // iwLs_a iwLs_b: W node
  double iW_GL[MHD_NMAX][MHD_LMAX];  // iwG_a iwLs_b: N_x node
  double iW_LG[MHD_LMAX][MHD_NMAX];  // iwLs_a iwG_b: N_y node
};

__constant__ MTab c_mtab[8];

void upload_mag_tables(int slot, const Tab* h, cudaError_t* err) {
  MTab m;
  memcpy(m.wp, h->wp, sizeof m.wp);
  memcpy(m.wL, h->wL, sizeof m.wL);
  memcpy(m.wG, h->wG, sizeof m.wG);
  memcpy(m.ML, h->ML, sizeof m.ML);
  memcpy(m.dL_G, h->dL_G, sizeof m.dL_G);
  memcpy(m.G_L, h->G_L, sizeof m.G_L);
  memcpy(m.M_G, h->M_G, sizeof m.M_G);
  memcpy(m.M_L, h->M_L, sizeof m.M_L);
  memcpy(m.P_G, h->P_G, sizeof m.P_G);
  memcpy(m.P_L, h->P_L, sizeof m.P_L);
  memcpy(m.dL_M, h->dL_M, sizeof m.dL_M);
  memcpy(m.G_M, h->G_M, sizeof m.G_M);
  memcpy(m.L_P, h->L_P, sizeof m.L_P);
  memcpy(m.G_P, h->G_P, sizeof m.G_P);
  memcpy(m.WG_P, h->WG_P, sizeof m.WG_P);
  memcpy(m.WL_P, h->WL_P, sizeof m.WL_P);
  memcpy(m.iwLs, h->iwLs, sizeof m.iwLs);
  memcpy(m.iwG, h->iwG, sizeof m.iwG);
  for (int j = 0; j < MHD_NMAX; ++j)
    for (int b = 0; b < MHD_LMAX; ++b) {
      m.wdL_G[j][b] = h->wG[j] * h->dL_G[j][b];
      m.W_GL[j][b] = h->wG[j] * h->wL[b];
    }
  for (int a = 0; a < MHD_LMAX; ++a)
    for (int b = 0; b < MHD_NMAX; ++b) m.W_LG[a][b] = h->wL[a] * h->wG[b];
  for (int a = 0; a < MHD_LMAX; ++a)
    for (int b = 0; b < MHD_LMAX; ++b) {
      m.W_LL[a][b] = h->wL[a] * h->wL[b];
      m.iW_LL[a][b] = h->iwLs[a] * h->iwLs[b];
    }
  for (int a = 0; a < MHD_NMAX; ++a)
    for (int b = 0; b < MHD_LMAX; ++b) m.iW_GL[a][b] = h->iwG[a] * h->iwLs[b];
  for (int a = 0; a < MHD_LMAX; ++a)
    for (int b = 0; b < MHD_NMAX; ++b) m.iW_LG[a][b] = h->iwLs[a] * h->iwG[b];
  *err = cudaMemcpyToSymbol(c_mtab, &m, sizeof(MTab), slot * sizeof(MTab));
}

template <int P, int KM, int EBv = mag_tile_eb(0)>
struct MD {
  static constexpr int n = P + 1, n2 = n * n, mm = KM + 1, mL = KM + 2;
  static constexpr int NX = mm * mL;   // N_x family / Y-type arrays: a < mm (Gauss x), b < mL (GLL y)
  static constexpr int NY = mL * mm;   // N_y family / X-type arrays: a < mL (GLL x), b < mm (Gauss y)
  static constexpr int NW = mL * mL;   // W family
  static constexpr int NZ = mm * mm;   // owned DOFs / B_z
  static constexpr int EB = EBv;       // elements per block (autotuned variant)
  static constexpr int TH = 256;       // threads per block
  static constexpr int SLOT = P - 1 + KM;
  // k = p - 1: the GLL(k+1) nodes of the auxiliary families are the DG nodes
  // (the same rule, so the same doubles), and the tables between them, P_L and
  // L_P, are exactly the identity; every pass through them is skipped (a copy
  // gives the same bits as the FMA chain it replaces: one term 1 * x, the
  // others 0 * x).
  static constexpr bool LID = mL == n;
};

#define FLAT(ITEMS) for (int idx = threadIdx.x; idx < D::EB * (ITEMS); idx += blockDim.x)
#define SM(off, it) sm[(size_t)((off) + (it)) * D::EB + e]

// ---- assembly of closure values from element loads ----------------------------
// The sums of the element loads at a closure node (the *_sum helpers, in one
// canonical order: south-west contribution first) and the assembled values
// (sum times 1 / (Jdet times the assembled lumped weight)).
// W-type closure node (a, b), a, b < mL, of element (ex, ey).
template <int P, int KM>
__device__ __forceinline__ double assemble_W_sum(const double* __restrict__ Lz, int ex, int ey, int a, int b,
                                                 const Mesh& M) {
  using D = MD<P, KM>;
  int ox = ex, oy = ey, ao = a, bo = b;
  if (a == D::mL - 1) { ox = wrap(ex + 1, M.nx); ao = 0; }
  if (b == D::mL - 1) { oy = wrap(ey + 1, M.ny); bo = 0; }
  const int wx = wrap(ox - 1, M.nx), sy = wrap(oy - 1, M.ny);
  double v = 0.0;
  const size_t KW = (size_t)M.K * D::NW;
  if (ao == 0 && bo == 0) v += Lz[MHD_CHK((size_t)(sy * M.nx + wx) * D::NW + (D::mL - 1) * D::mL + (D::mL - 1), KW)];
  if (bo == 0) v += Lz[MHD_CHK((size_t)(sy * M.nx + ox) * D::NW + (D::mL - 1) * D::mL + ao, KW)];
  if (ao == 0) v += Lz[MHD_CHK((size_t)(oy * M.nx + wx) * D::NW + bo * D::mL + (D::mL - 1), KW)];
  v += Lz[MHD_CHK((size_t)(oy * M.nx + ox) * D::NW + bo * D::mL + ao, KW)];
  return v;
}
template <int P, int KM>
__device__ __forceinline__ double assemble_W(const double* __restrict__ Lz, int ex, int ey, int a, int b,
                                             const Mesh& M, double iJ) {
  using D = MD<P, KM>;
  const MTab& T = c_mtab[D::SLOT];
  const int ao = a == D::mL - 1 ? 0 : a, bo = b == D::mL - 1 ? 0 : b;
  return assemble_W_sum<P, KM>(Lz, ex, ey, a, b, M) * (iJ * T.iW_LL[ao][bo]);
}

// Y-type (N_x) closure node (a < mm, b < mL).
template <int P, int KM>
__device__ __forceinline__ double assemble_Nx_sum(const double* __restrict__ Lx, int ex, int ey, int a, int b,
                                                  const Mesh& M) {
  using D = MD<P, KM>;
  int oy = ey, bo = b;
  if (b == D::mL - 1) { oy = wrap(ey + 1, M.ny); bo = 0; }
  const int sy = wrap(oy - 1, M.ny);
  double v = 0.0;
  const size_t KX = (size_t)M.K * D::NX;
  if (bo == 0) v += Lx[MHD_CHK((size_t)(sy * M.nx + ex) * D::NX + (D::mL - 1) * D::mm + a, KX)];
  v += Lx[MHD_CHK((size_t)(oy * M.nx + ex) * D::NX + bo * D::mm + a, KX)];
  return v;
}
template <int P, int KM>
__device__ __forceinline__ double assemble_Nx(const double* __restrict__ Lx, int ex, int ey, int a, int b,
                                              const Mesh& M, double iJ) {
  using D = MD<P, KM>;
  const MTab& T = c_mtab[D::SLOT];
  return assemble_Nx_sum<P, KM>(Lx, ex, ey, a, b, M) * (iJ * T.iW_GL[a][b == D::mL - 1 ? 0 : b]);
}

// X-type (N_y) closure node (a < mL, b < mm).
template <int P, int KM>
__device__ __forceinline__ double assemble_Ny_sum(const double* __restrict__ Ly, int ex, int ey, int a, int b,
                                                  const Mesh& M) {
  using D = MD<P, KM>;
  int ox = ex, ao = a;
  if (a == D::mL - 1) { ox = wrap(ex + 1, M.nx); ao = 0; }
  const int wx = wrap(ox - 1, M.nx);
  double v = 0.0;
  const size_t KY = (size_t)M.K * D::NY;
  if (ao == 0) v += Ly[MHD_CHK((size_t)(ey * M.nx + wx) * D::NY + b * D::mL + (D::mL - 1), KY)];
  v += Ly[MHD_CHK((size_t)(ey * M.nx + ox) * D::NY + b * D::mL + ao, KY)];
  return v;
}
template <int P, int KM>
__device__ __forceinline__ double assemble_Ny(const double* __restrict__ Ly, int ex, int ey, int a, int b,
                                              const Mesh& M, double iJ) {
  using D = MD<P, KM>;
  const MTab& T = c_mtab[D::SLOT];
  return assemble_Ny_sum<P, KM>(Ly, ex, ey, a, b, M) * (iJ * T.iW_LG[a == D::mL - 1 ? 0 : a][b]);
}

// Per-block factors of the closure families in the order of their items
// (N_x, then N_y, then W): the assembly factor 1 / (Jdet times the assembled
// lumped weight), and (lumped) Jdet times the element's lumped weight.  Both
// are the same doubles the per-item products would give.
template <int P, int KM>
__device__ __forceinline__ void closure_factors(double* __restrict__ af, double* __restrict__ pw, const Mesh& M) {
  using D = MD<P, KM>;
  const MTab& T = c_mtab[D::SLOT];
  for (int t = threadIdx.x; t < D::NX + D::NY + D::NW; t += blockDim.x) {
    double f, w;
    if (t < D::NX) {
      const int a = t % D::mm, b = t / D::mm;
      f = M.iJ * T.iW_GL[a][b == D::mL - 1 ? 0 : b];
      w = M.Jdet * T.W_GL[a][b];
    } else if (t < D::NX + D::NY) {
      const int r = t - D::NX, a = r % D::mL, b = r / D::mL;
      f = M.iJ * T.iW_LG[a == D::mL - 1 ? 0 : a][b];
      w = M.Jdet * T.W_LG[a][b];
    } else {
      const int r = t - D::NX - D::NY, a = r % D::mL, b = r / D::mL;
      f = M.iJ * T.iW_LL[a == D::mL - 1 ? 0 : a][b == D::mL - 1 ? 0 : b];
      w = M.Jdet * T.W_LL[a][b];
    }
    af[t] = f;
    if (pw) pw[t] = w;
  }
}

// B closure loads: Bx (X-type, [b < mm][a < mL]) and By (Y-type, [b < mL][a < mm]).
template <int P, int KM>
__device__ __forceinline__ double closure_Bx(const double* __restrict__ Bx, int ex, int ey, int a, int b,
                                             const Mesh& M) {
  using D = MD<P, KM>;
  if (a == D::mL - 1) return Bx[MHD_CHK((size_t)(ey * M.nx + wrap(ex + 1, M.nx)) * D::NZ + b * D::mm, (size_t)M.K * D::NZ)];
  return Bx[MHD_CHK((size_t)(ey * M.nx + ex) * D::NZ + b * D::mm + a, (size_t)M.K * D::NZ)];
}
template <int P, int KM>
__device__ __forceinline__ double closure_By(const double* __restrict__ By, int ex, int ey, int a, int b,
                                             const Mesh& M) {
  using D = MD<P, KM>;
  if (b == D::mL - 1) return By[MHD_CHK((size_t)(wrap(ey + 1, M.ny) * M.nx + ex) * D::NZ + a, (size_t)M.K * D::NZ)];
  return By[MHD_CHK((size_t)(ey * M.nx + ex) * D::NZ + b * D::mm + a, (size_t)M.K * D::NZ)];
}

// ============================ k_mag_J ==========================================
template <int P, int KM>
struct LJ_ {  // per-element shared-memory offsets (doubles)
  using D = MD<P, KM>;
  static constexpr int BX = 0, BY = BX + D::NY, BZ = BY + D::NX;
  static constexpr int T1 = BZ + D::NZ;          // [j < mm][a < mL]
  static constexpr int T2 = T1 + D::mm * D::mL;  // [b < mL][i < mm]
  static constexpr int TA = T2 + D::mL * D::mm;  // Bz rows to Gauss x
  static constexpr int BZG = TA + D::NZ;         // Bz at Gauss(k)^2: [d][a]
  static constexpr int SIZE = BZG + D::NZ;
};

template <int P, int KM, int EBv = mag_tile_eb(0), bool R2 = false>
__global__ void __launch_bounds__(256) k_mag_J(const double* __restrict__ Bx, const double* __restrict__ By,
                                               const double* __restrict__ Bz, double* __restrict__ LJx,
                                               double* __restrict__ LJy, double* __restrict__ LJz, Mesh M) {
  using D = MD<P, KM, EBv>;
  using O = LJ_<P, KM>;
  const MTab& T = c_mtab[D::SLOT];
  extern __shared__ double sm[];
  const int k0 = blockIdx.x * D::EB;
  // 2D2V (R2): B_z = 0, so only the W loads of J_z are formed
  constexpr int I1 = D::NY + D::NX + (R2 ? 0 : D::NZ);
  FLAT(I1) {
    int it = idx / D::EB, e = idx % D::EB, k = min(k0 + e, M.K - 1);
    int ex = k % M.nx, ey = k / M.nx;
    if (it < D::NY) SM(O::BX, it) = closure_Bx<P, KM>(Bx, ex, ey, it % D::mL, it / D::mL, M);
    else if (it < D::NY + D::NX) { it -= D::NY; SM(O::BY, it) = closure_By<P, KM>(By, ex, ey, it % D::mm, it / D::mm, M); }
    else { it -= D::NY + D::NX; SM(O::BZ, it) = Bz[MHD_CHK((size_t)k * D::NZ + it, (size_t)M.K * D::NZ)]; }
  }
  __syncthreads();
  constexpr int I2 = D::mm * D::mL + D::mL * D::mm + (R2 ? 0 : D::NZ);
  FLAT(I2) {
    int it = idx / D::EB, e = idx % D::EB;
    if (it < D::mm * D::mL) {
      int j = it / D::mL, a = it % D::mL;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < D::mL; ++i) s = fma(SM(O::BX, j * D::mL + i), T.ML[i][a], s);
      SM(O::T1, it) = s;
    } else if (it < 2 * D::mm * D::mL) {
      it -= D::mm * D::mL;
      int b = it / D::mm, i = it % D::mm;
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < D::mL; ++j) s = fma(T.ML[j][b], SM(O::BY, j * D::mm + i), s);
      SM(O::T2, it) = s;
    } else {
      it -= 2 * D::mm * D::mL;
      int r = it / D::mm, a = it % D::mm;
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) s = fma(T.M_G[a][c], SM(O::BZ, r * D::mm + c), s);
      SM(O::TA, it) = s;
    }
  }
  __syncthreads();
  const double cy = 2.0 * M.ihy * M.Jdet, cx = 2.0 * M.ihx * M.Jdet;
  constexpr int I3 = D::NW + (R2 ? 0 : D::NZ);
  FLAT(I3) {
    int it = idx / D::EB, e = idx % D::EB, k = k0 + e;
    if (it < D::NW) {
      int b = it / D::mL, a = it % D::mL;
      double z1 = 0.0, z2 = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) {
        z1 = fma(T.wdL_G[j][b], SM(O::T1, j * D::mL + a), z1);
        z2 = fma(T.wdL_G[j][a], SM(O::T2, b * D::mm + j), z2);
      }
      if (k < M.K) LJz[MHD_CHK((size_t)k * D::NW + it, (size_t)M.K * D::NW)] = fma(cy, z1, -cx * z2);
    } else {
      it -= D::NW;
      int d = it / D::mm, a = it % D::mm;
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < D::mm; ++r) s = fma(T.M_G[d][r], SM(O::TA, r * D::mm + a), s);
      SM(O::BZG, it) = s;
    }
  }
  __syncthreads();
  constexpr int I4 = R2 ? 0 : D::NX + D::NY;
  FLAT(I4) {
    int it = idx / D::EB, e = idx % D::EB, k = k0 + e;
    if (k >= M.K) continue;
    if (it < D::NX) {  // J_x: a < mm (Gauss x), b < mL
      int b = it / D::mm, a = it % D::mm;
      double s = 0.0;
#pragma unroll
      for (int d = 0; d < D::mm; ++d) s = fma(T.wdL_G[d][b], SM(O::BZG, d * D::mm + a), s);
      LJx[MHD_CHK((size_t)k * D::NX + it, (size_t)M.K * D::NX)] = -cy * T.wG[a] * s;
    } else {  // J_y: a < mL (GLL x), b < mm
      it -= D::NX;
      int b = it / D::mL, a = it % D::mL;
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) s = fma(T.wdL_G[c][a], SM(O::BZG, b * D::mm + c), s);
      LJy[MHD_CHK((size_t)k * D::NY + it, (size_t)M.K * D::NY)] = cx * T.wG[b] * s;
    }
  }
}

// ============================ k_mag_E ==========================================
template <int P, int KM>
struct LE_ {  // per-element shared-memory offsets (doubles), with region reuse
  using D = MD<P, KM>;
  // region A: closures (live through the pointwise stage; J also in the resistive stage)
  static constexpr int JX = 0, JY = JX + D::NX, JZ = JY + D::NY, BX = JZ + D::NW, BY = BX + D::NY, BZ = BY + D::NX;
  static constexpr int ETA = BZ + D::NZ;
  static constexpr int RB = ETA + 1;
  // region B: first passes (dead after the second ones; BYL is read by the pointwise stage),
  // then the transposed passes.  Each velocity component takes, per family, the cheaper pass
  // order, and a first pass is shared where two families share that direction's nodes:
  // u_x rows to GLL(k+1) x (N_y, W), u_y columns to GLL(k+1) y (N_x, W), u_z rows to Gauss x
  // (N_x) and columns to Gauss y (N_y)
  static constexpr int UGZ = RB;                         // u_z rows to Gauss x: [j < n][a < mm]
  static constexpr int ULX = UGZ + D::n * D::mm;         // u_x rows to GLL(k+1) x: [j < n][a < mL]
  static constexpr int CYY = ULX + D::n * D::mL;         // u_y columns to GLL(k+1) y: [b < mL][i < n]
  static constexpr int CGZ = CYY + D::mL * D::n;         // u_z columns to Gauss y: [b < mm][i < n]
  static constexpr int BYL = CGZ + D::mm * D::n;         // By rows (GLL y) to GLL x (= By at W)
  static constexpr int BZG = BYL + D::NW;                // Bz rows to Gauss x
  static constexpr int BZC = BZG + D::NZ;                // Bz columns to Gauss y: [b < mm][a < mm]
  static constexpr int RB_END = BZC + D::NZ;
  // transposed passes of the Lorentz load: s_x (N_y and W, GLL(k+1) x) y-first into VX [j][a];
  // s_y (N_x and W, GLL(k+1) y) x-first into HY [b][i]; s_z: N_x y-first into VZ1 [j][a],
  // N_y x-first into HZ [b][i] (each family in its cheaper order)
  static constexpr int VX = RB, HY = VX + D::n * D::mL, VZ1 = HY + D::mL * D::n, HZ = VZ1 + D::n * D::mm,
                       V_END = HZ + D::mm * D::n;
  static constexpr int RC = RB_END > V_END ? RB_END : V_END;
  // region C: values at the auxiliary families; Lorentz products overwrite them in place;
  // the resistive stage reuses it afterwards
  static constexpr int UNX = RC, UNY = UNX + 2 * D::NX, UW = UNY + 2 * D::NY;
  static constexpr int BXNX = UW + 2 * D::NW, BZNX = BXNX + D::NX, BYNY = BZNX + D::NX, BZNY = BYNY + D::NY;
  static constexpr int BXW = BZNY + D::NY, BZW = BXW + D::NW, RC_END = BZW + D::NW;
  static constexpr int TQ = RC, JQ = TQ + 3 * D::n * D::mL, RQ_END = JQ + 3 * D::n2;
  // per-block factors (closure_factors: 2 (NX + NY + NW) doubles, then the
  // lumped DG-node masses Jdet w_i w_j) in slots after the per-element
  // regions; at least 8 elements per block
  static constexpr int FAC = RC_END > RQ_END ? RC_END : RQ_END;
  static constexpr int SIZE = FAC + (2 * (D::NX + D::NY + D::NW) + D::n2 + 7) / 8;
};

// mode 0: write du, de (residual test hook); mode 1: SSP combination into (uo, eo);
// mode 2: raw Lorentz load only (adjoint, see magnetic_adjoint.inc).
template <int P, int KM, int MODE, int EBv = mag_tile_eb(0), bool R2 = false>
__global__ void __launch_bounds__(256) k_mag_E(
    const double* __restrict__ LJx, const double* __restrict__ LJy, const double* __restrict__ LJz,
    const double* __restrict__ Bx, const double* __restrict__ By, const double* __restrict__ Bz,
    const double* __restrict__ u, const double* __restrict__ e_in, const double* __restrict__ rho,
    const double* __restrict__ eta, const double* u0, const double* e0, double* uo, double* eo,
    double* __restrict__ LEx, double* __restrict__ LEy, double* __restrict__ LEz, Mesh M,
    const double* __restrict__ dtp, double dtfac, double ca, double cb, int first, int resistive) {
  using D = MD<P, KM, EBv>;
  using O = LE_<P, KM>;
  const MTab& T = c_mtab[D::SLOT];
  extern __shared__ double sm[];
  const int k0 = blockIdx.x * D::EB;
  const size_t N = (size_t)M.K * D::n2;
  static_assert(D::EB >= 8, "per-block factor slots assume at least 8 elements per block");
  double* const sAF = sm + (size_t)O::FAC * D::EB;  // assembly factors [NX | NY | NW]
  double* const sPW = sAF + D::NX + D::NY + D::NW;  // lumped weights Jdet w [NX | NY | NW]
  double* const sMW = sPW + D::NX + D::NY + D::NW;  // DG-node masses Jdet w_i w_j [n2]
  closure_factors<P, KM>(sAF, sPW, M);
  for (int t = threadIdx.x; t < D::n2; t += blockDim.x) sMW[t] = M.Jdet * T.wp[t % D::n] * T.wp[t / D::n];
  __syncthreads();
  // stage 1: J closure (assembled), B closure, eta (2D2V: J_z, B_x, B_y and eta only)
  constexpr int I1 = (R2 ? 0 : D::NX + D::NY) + D::NW + D::NY + D::NX + (R2 ? 0 : D::NZ) + 1;
  FLAT(I1) {
    int it = idx / D::EB, e = idx % D::EB, k = min(k0 + e, M.K - 1);
    int ex = k % M.nx, ey = k / M.nx;
    if constexpr (!R2) {
      if (it < D::NX) { SM(O::JX, it) = assemble_Nx_sum<P, KM>(LJx, ex, ey, it % D::mm, it / D::mm, M) * sAF[it]; continue; }
      it -= D::NX;
      if (it < D::NY) { SM(O::JY, it) = assemble_Ny_sum<P, KM>(LJy, ex, ey, it % D::mL, it / D::mL, M) * sAF[D::NX + it]; continue; }
      it -= D::NY;
    }
    if (it < D::NW) {
      SM(O::JZ, it) = assemble_W_sum<P, KM>(LJz, ex, ey, it % D::mL, it / D::mL, M) * sAF[D::NX + D::NY + it];
      continue;
    }
    it -= D::NW;
    if (it < D::NY) { SM(O::BX, it) = closure_Bx<P, KM>(Bx, ex, ey, it % D::mL, it / D::mL, M); continue; }
    it -= D::NY;
    if (it < D::NX) { SM(O::BY, it) = closure_By<P, KM>(By, ex, ey, it % D::mm, it / D::mm, M); continue; }
    it -= D::NX;
    if constexpr (!R2) {
      if (it < D::NZ) { SM(O::BZ, it) = Bz[MHD_CHK((size_t)k * D::NZ + it, (size_t)M.K * D::NZ)]; continue; }
    }
    SM(O::ETA, 0) = resistive ? eta[MHD_CHK(k, M.K)] : 0.0;
  }
  __syncthreads();
  // stage 2: first passes (u read straight from global memory); only what the
  // cross products need: E_x = -(u_y B_z - u_z B_y) at N_x, E_y = -(u_z B_x -
  // u_x B_z) at N_y, E_z = -(u_x B_y - u_y B_x) at W
  constexpr int NUZ = R2 ? 0 : D::n * D::mm, NUL = 2 * D::n * D::mL;
  constexpr int I2 = 2 * NUZ + NUL + D::NW + (R2 ? 0 : 2 * D::NZ);
  FLAT(I2) {
    int it = idx / D::EB, e = idx % D::EB, k = min(k0 + e, M.K - 1);
    if constexpr (!R2) {
      if (it < NUZ) {  // u_z rows to Gauss x
        int j = it / D::mm, a = it % D::mm;
        const double* ur = u + MHD_CHK(2 * N + (size_t)k * D::n2 + j * D::n, 3 * N - D::n + 1);
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < D::n; ++i) v = fma(T.P_G[a][i], ur[i], v);
        SM(O::UGZ, it) = v;
        continue;
      }
      it -= NUZ;
    }
    if (it < D::n * D::mL) {  // u_x rows to GLL(k+1) x
      int j = it / D::mL, a = it % D::mL;
      const double* ur = u + MHD_CHK((size_t)k * D::n2 + j * D::n, 3 * N - D::n + 1);
      double v = 0.0;
      if constexpr (D::LID) v = ur[a];
      else {
#pragma unroll
        for (int i = 0; i < D::n; ++i) v = fma(T.P_L[a][i], ur[i], v);
      }
      SM(O::ULX, it) = v;
      continue;
    }
    it -= D::n * D::mL;
    if (it < D::mL * D::n) {  // u_y columns to GLL(k+1) y
      int b = it / D::n, i = it % D::n;
      const double* uc = u + MHD_CHK(N + (size_t)k * D::n2 + i, 3 * N - (D::n - 1) * D::n);
      double v = 0.0;
      if constexpr (D::LID) v = uc[b * D::n];
      else {
#pragma unroll
        for (int j = 0; j < D::n; ++j) v = fma(T.P_L[b][j], uc[j * D::n], v);
      }
      SM(O::CYY, it) = v;
      continue;
    }
    it -= D::mL * D::n;
    if constexpr (!R2) {
      if (it < NUZ) {  // u_z columns to Gauss y
        int b = it / D::n, i = it % D::n;
        const double* uc = u + MHD_CHK(2 * N + (size_t)k * D::n2 + i, 3 * N - (D::n - 1) * D::n);
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < D::n; ++j) v = fma(T.P_G[b][j], uc[j * D::n], v);
        SM(O::CGZ, it) = v;
        continue;
      }
      it -= NUZ;
    }
    if (it < D::NW) {  // By rows (GLL y) to GLL x
      int j = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int i = 0; i < D::mm; ++i) v = fma(T.G_L[a][i], SM(O::BY, j * D::mm + i), v);
      SM(O::BYL, it) = v;
      continue;
    }
    it -= D::NW;
    if constexpr (!R2) {
      if (it < D::NZ) {  // Bz rows to Gauss x
        int j = it / D::mm, a = it % D::mm;
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < D::mm; ++i) v = fma(T.M_G[a][i], SM(O::BZ, j * D::mm + i), v);
        SM(O::BZG, it) = v;
        continue;
      }
      it -= D::NZ;
      {  // Bz columns to Gauss y (for N_y: y first, then x)
        int b = it / D::mm, a = it % D::mm;
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < D::mm; ++j) v = fma(T.M_G[b][j], SM(O::BZ, j * D::mm + a), v);
        SM(O::BZC, it) = v;
      }
    }
  }
  __syncthreads();
  // stage 3: second passes to the auxiliary families
  constexpr int I3 = (R2 ? 0 : 2 * D::NX + 2 * D::NY) + 2 * D::NW + (R2 ? 0 : D::NX + D::NY) + D::NW;
  FLAT(I3) {
    int it = idx / D::EB, e = idx % D::EB;
    if constexpr (!R2) {
      if (it < D::NX) {  // u_y at N_x (a < mm Gauss x, b < mL): x-pass of the GLL(k+1)-y columns
        int b = it / D::mm, a = it % D::mm;
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < D::n; ++i) v = fma(T.P_G[a][i], SM(O::CYY, b * D::n + i), v);
        SM(O::UNX, it) = v;
        continue;
      }
      if (it < 2 * D::NX) {  // u_z at N_x: y-pass of the Gauss-x rows
        const int r = it - D::NX, b = r / D::mm, a = r % D::mm;
        double v = 0.0;
        if constexpr (D::LID) v = SM(O::UGZ, b * D::mm + a);
        else {
#pragma unroll
          for (int j = 0; j < D::n; ++j) v = fma(T.P_L[b][j], SM(O::UGZ, j * D::mm + a), v);
        }
        SM(O::UNX, it) = v;
        continue;
      }
      it -= 2 * D::NX;
      if (it < D::NY) {  // u_x at N_y (a < mL, b < mm Gauss y): y-pass of the GLL(k+1)-x rows
        int b = it / D::mL, a = it % D::mL;
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < D::n; ++j) v = fma(T.P_G[b][j], SM(O::ULX, j * D::mL + a), v);
        SM(O::UNY, it) = v;
        continue;
      }
      if (it < 2 * D::NY) {  // u_z at N_y: x-pass of the Gauss-y columns
        const int r = it - D::NY, b = r / D::mL, a = r % D::mL;
        double v = 0.0;
        if constexpr (D::LID) v = SM(O::CGZ, b * D::n + a);
        else {
#pragma unroll
          for (int i = 0; i < D::n; ++i) v = fma(T.P_L[a][i], SM(O::CGZ, b * D::n + i), v);
        }
        SM(O::UNY, it) = v;
        continue;
      }
      it -= 2 * D::NY;
    }
    if (it < D::NW) {  // u_x at W: y-pass of the GLL(k+1)-x rows
      int b = it / D::mL, a = it % D::mL;
      double v = 0.0;
      if constexpr (D::LID) v = SM(O::ULX, b * D::mL + a);
      else {
#pragma unroll
        for (int j = 0; j < D::n; ++j) v = fma(T.P_L[b][j], SM(O::ULX, j * D::mL + a), v);
      }
      SM(O::UW, it) = v;
      continue;
    }
    if (it < 2 * D::NW) {  // u_y at W: x-pass of the GLL(k+1)-y columns
      const int r = it - D::NW, b = r / D::mL, a = r % D::mL;
      double v = 0.0;
      if constexpr (D::LID) v = SM(O::CYY, b * D::n + a);
      else {
#pragma unroll
        for (int i = 0; i < D::n; ++i) v = fma(T.P_L[a][i], SM(O::CYY, b * D::n + i), v);
      }
      SM(O::UW, it) = v;
      continue;
    }
    it -= 2 * D::NW;
    if constexpr (!R2) {
      if (it < D::NX) {  // Bz at N_x: GLL(k) y -> GLL(k+1) y
        int b = it / D::mm, a = it % D::mm;
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < D::mm; ++j) v = fma(T.M_L[b][j], SM(O::BZG, j * D::mm + a), v);
        SM(O::BZNX, it) = v;
        continue;
      }
      it -= D::NX;
      if (it < D::NY) {  // Bz at N_y: the Gauss-y columns to GLL(k+1) x
        int b = it / D::mL, a = it % D::mL;
        double v = 0.0;
#pragma unroll
        for (int c = 0; c < D::mm; ++c) v = fma(T.M_L[a][c], SM(O::BZC, b * D::mm + c), v);
        SM(O::BZNY, it) = v;
        continue;
      }
      it -= D::NY;
    }
    {  // Bx at W: Gauss y -> GLL y
      int b = it / D::mL, a = it % D::mL;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < D::mm; ++j) v = fma(T.G_L[b][j], SM(O::BX, j * D::mL + a), v);
      SM(O::BXW, it) = v;
    }
  }
  __syncthreads();
  // stage 4: pointwise E loads (lumped weights); Lorentz products overwrite the u values in place
  const double Jd = M.Jdet;
  constexpr int I4 = (R2 ? 0 : D::NX + D::NY) + D::NW;
  FLAT(I4) {
    int it = idx / D::EB, e = idx % D::EB, k = k0 + e;
    if (!R2 && it < D::NX) {
      const double w = sPW[it];
      double by_ = SM(O::BY, it), bz_ = SM(O::BZNX, it), jx_ = SM(O::JX, it);
      double uy = SM(O::UNX, it), uz = SM(O::UNX, D::NX + it);
      if (k < M.K) LEx[MHD_CHK((size_t)k * D::NX + it, (size_t)M.K * D::NX)] = w * fma(uz, by_, -uy * bz_);
      const double wj = w * jx_;
      SM(O::UNX, it) = -wj * bz_;         // s_y contribution
      SM(O::UNX, D::NX + it) = wj * by_;  // s_z contribution
    } else if (!R2 && it < D::NX + D::NY) {
      it -= D::NX;
      const double w = sPW[D::NX + it];
      double bx_ = SM(O::BX, it), bz_ = SM(O::BZNY, it), jy_ = SM(O::JY, it);
      double ux = SM(O::UNY, it), uz = SM(O::UNY, D::NY + it);
      if (k < M.K) LEy[MHD_CHK((size_t)k * D::NY + it, (size_t)M.K * D::NY)] = w * fma(ux, bz_, -uz * bx_);
      const double wj = w * jy_;
      SM(O::UNY, it) = wj * bz_;           // s_x
      SM(O::UNY, D::NY + it) = -wj * bx_;  // s_z
    } else {
      if constexpr (!R2) it -= D::NX + D::NY;
      const double w = sPW[D::NX + D::NY + it];
      double bx_ = SM(O::BXW, it), by_ = SM(O::BYL, it), jz_ = SM(O::JZ, it);
      double ux = SM(O::UW, it), uy = SM(O::UW, D::NW + it);
      if (k < M.K) LEz[MHD_CHK((size_t)k * D::NW + it, (size_t)M.K * D::NW)] = w * fma(uy, bx_, -ux * by_);
      const double wj = w * jz_;
      SM(O::UW, it) = -wj * by_;          // s_x
      SM(O::UW, D::NW + it) = wj * bx_;   // s_y
    }
  }
  __syncthreads();
  // stage 5: first transposed passes of the Lorentz load (into region B)
  constexpr int I5 = 2 * D::n * D::mL + (R2 ? 0 : 2 * D::n * D::mm);
  FLAT(I5) {
    int it = idx / D::EB, e = idx % D::EB;
    if (it < D::n * D::mL) {  // s_x: y-pass of N_y (Gauss y) and W (GLL y) onto the DG rows j
      int j = it / D::mL, a = it % D::mL;
      // at k = p - 1 the W part is a copy: it starts the chain
      double v = D::LID ? SM(O::UW, j * D::mL + a) : 0.0;
      if constexpr (!R2) {
#pragma unroll
        for (int b = 0; b < D::mm; ++b) v = fma(T.P_G[b][j], SM(O::UNY, b * D::mL + a), v);
      }
      if constexpr (!D::LID) {
#pragma unroll
        for (int b = 0; b < D::mL; ++b) v = fma(T.P_L[b][j], SM(O::UW, b * D::mL + a), v);
      }
      SM(O::VX, it) = v;
      continue;
    }
    it -= D::n * D::mL;
    if (it < D::mL * D::n) {  // s_y: x-pass of N_x (Gauss x) and W (GLL x) onto the DG columns i, rows b
      int b = it / D::n, i = it % D::n;
      double v = D::LID ? SM(O::UW, D::NW + b * D::mL + i) : 0.0;
      if constexpr (!R2) {
#pragma unroll
        for (int a = 0; a < D::mm; ++a) v = fma(T.P_G[a][i], SM(O::UNX, b * D::mm + a), v);
      }
      if constexpr (!D::LID) {
#pragma unroll
        for (int a = 0; a < D::mL; ++a) v = fma(T.P_L[a][i], SM(O::UW, D::NW + b * D::mL + a), v);
      }
      SM(O::HY, it) = v;
      continue;
    }
    it -= D::mL * D::n;
    if constexpr (!R2) {
      if (it < D::n * D::mm) {  // s_z from N_x: y-pass (GLL y) onto the DG rows j
        int j = it / D::mm, a = it % D::mm;
        double v = 0.0;
        if constexpr (D::LID) v = SM(O::UNX, D::NX + j * D::mm + a);
        else {
#pragma unroll
          for (int b = 0; b < D::mL; ++b) v = fma(T.P_L[b][j], SM(O::UNX, D::NX + b * D::mm + a), v);
        }
        SM(O::VZ1, it) = v;
        continue;
      }
      it -= D::n * D::mm;
      {  // s_z from N_y: x-pass (GLL x) onto the DG columns i, rows b (Gauss y)
        int b = it / D::n, i = it % D::n;
        double v = 0.0;
        if constexpr (D::LID) v = SM(O::UNY, D::NY + b * D::mL + i);
        else {
#pragma unroll
          for (int a = 0; a < D::mL; ++a) v = fma(T.P_L[a][i], SM(O::UNY, D::NY + b * D::mL + a), v);
        }
        SM(O::HZ, it) = v;
      }
    }
  }
  __syncthreads();
  // stage 5b (resistive only): J_h at the DG nodes and the resistive loads
  if (resistive) {
    constexpr int IR1 = (R2 ? 0 : D::mL * D::n + D::mm * D::n) + D::mL * D::n;
    FLAT(IR1) {
      int it = idx / D::EB, e = idx % D::EB;
      if (SM(O::ETA, 0) == 0.0) continue;
      if constexpr (R2) it += D::mL * D::n + D::mm * D::n;  // J_z only
      if (it < D::mL * D::n) {
        int b = it / D::n, i = it % D::n;
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < D::mm; ++a) v = fma(T.G_P[i][a], SM(O::JX, b * D::mm + a), v);
        SM(O::TQ, it) = v;
      } else if (it < D::mL * D::n + D::mm * D::n) {
        it -= D::mL * D::n;
        int b = it / D::n, i = it % D::n;
        double v = 0.0;
        if constexpr (D::LID) v = SM(O::JY, b * D::mL + i);
        else {
#pragma unroll
          for (int a = 0; a < D::mL; ++a) v = fma(T.L_P[i][a], SM(O::JY, b * D::mL + a), v);
        }
        SM(O::TQ, D::n * D::mL + it) = v;
      } else {
        it -= D::mL * D::n + D::mm * D::n;
        int b = it / D::n, i = it % D::n;
        double v = 0.0;
        if constexpr (D::LID) v = SM(O::JZ, b * D::mL + i);
        else {
#pragma unroll
          for (int a = 0; a < D::mL; ++a) v = fma(T.L_P[i][a], SM(O::JZ, b * D::mL + a), v);
        }
        SM(O::TQ, 2 * D::n * D::mL + it) = v;
      }
    }
    __syncthreads();
    constexpr int IR2 = (R2 ? 1 : 3) * D::n2;
    FLAT(IR2) {
      int it = idx / D::EB, e = idx % D::EB;
      if (SM(O::ETA, 0) == 0.0) continue;
      if constexpr (R2) it += 2 * D::n2;  // J_z only
      int d = it / D::n2, q = it % D::n2, j = q / D::n, i = q % D::n;
      double v = 0.0;
      if (d == 0) {
        if constexpr (D::LID) v = SM(O::TQ, j * D::n + i);
        else {
#pragma unroll
          for (int b = 0; b < D::mL; ++b) v = fma(T.L_P[j][b], SM(O::TQ, b * D::n + i), v);
        }
      } else if (d == 1) {
#pragma unroll
        for (int b = 0; b < D::mm; ++b) v = fma(T.G_P[j][b], SM(O::TQ, D::n * D::mL + b * D::n + i), v);
      } else {
        if constexpr (D::LID) v = SM(O::TQ, 2 * D::n * D::mL + j * D::n + i);
        else {
#pragma unroll
          for (int b = 0; b < D::mL; ++b) v = fma(T.L_P[j][b], SM(O::TQ, 2 * D::n * D::mL + b * D::n + i), v);
        }
      }
      SM(O::JQ, it) = v;
    }
    __syncthreads();
    // R_n = eta sum_q Jdet w_q J(x_q) phi_n(x_q), sum-factorised: x-pass of the
    // weighted DG-node values onto the basis in x (into the dead TQ area), then
    // y-pass, added to this element's own closure loads
    constexpr int IR3 = (R2 ? 0 : D::n * D::mm + D::n * D::mL) + D::n * D::mL;
    FLAT(IR3) {
      int it = idx / D::EB, e = idx % D::EB;
      if (SM(O::ETA, 0) == 0.0) continue;
      if constexpr (R2) it += D::n * D::mm + D::n * D::mL;  // W loads only
      if (it < D::n * D::mm) {  // N_x: basis g_a in x; rows j
        int j = it / D::mm, a = it % D::mm;
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < D::n; ++i) t = fma(T.WG_P[i][a], SM(O::JQ, j * D::n + i), t);
        SM(O::TQ, it) = t;
      } else if (it < D::n * D::mm + D::n * D::mL) {  // N_y: basis l^L_a in x
        it -= D::n * D::mm;
        int j = it / D::mL, a = it % D::mL;
        double t = 0.0;
        if constexpr (D::LID) t = T.WL_P[a][a] * SM(O::JQ, D::n2 + j * D::n + a);
        else {
#pragma unroll
          for (int i = 0; i < D::n; ++i) t = fma(T.WL_P[i][a], SM(O::JQ, D::n2 + j * D::n + i), t);
        }
        SM(O::TQ, D::n * D::mm + it) = t;
      } else {  // W: basis l^L_a in x
        it -= D::n * D::mm + D::n * D::mL;
        int j = it / D::mL, a = it % D::mL;
        double t = 0.0;
        if constexpr (D::LID) t = T.WL_P[a][a] * SM(O::JQ, 2 * D::n2 + j * D::n + a);
        else {
#pragma unroll
          for (int i = 0; i < D::n; ++i) t = fma(T.WL_P[i][a], SM(O::JQ, 2 * D::n2 + j * D::n + i), t);
        }
        SM(O::TQ, D::n * D::mm + D::n * D::mL + it) = t;
      }
    }
    __syncthreads();
    constexpr int IR4 = (R2 ? 0 : D::NX + D::NY) + D::NW;
    FLAT(IR4) {
      int it = idx / D::EB, e = idx % D::EB, k = k0 + e;
      const double et = SM(O::ETA, 0);
      if (et == 0.0 || k >= M.K) continue;
      if constexpr (R2) it += D::NX + D::NY;  // LEz only
      const double f = et * Jd;
      double r = 0.0;
      if (it < D::NX) {  // (a < mm, b < mL): y basis l^L_b
        int b = it / D::mm, a = it % D::mm;
        if constexpr (D::LID) r = T.WL_P[b][b] * SM(O::TQ, b * D::mm + a);
        else {
#pragma unroll
          for (int j = 0; j < D::n; ++j) r = fma(T.WL_P[j][b], SM(O::TQ, j * D::mm + a), r);
        }
        LEx[(size_t)k * D::NX + it] += f * r;
      } else if (it < D::NX + D::NY) {  // (a < mL, b < mm): y basis g_b
        it -= D::NX;
        int b = it / D::mL, a = it % D::mL;
#pragma unroll
        for (int j = 0; j < D::n; ++j) r = fma(T.WG_P[j][b], SM(O::TQ, D::n * D::mm + j * D::mL + a), r);
        LEy[(size_t)k * D::NY + it] += f * r;
      } else {  // W: y basis l^L_b
        it -= D::NX + D::NY;
        int b = it / D::mL, a = it % D::mL;
        if constexpr (D::LID) r = T.WL_P[b][b] * SM(O::TQ, D::n * D::mm + D::n * D::mL + b * D::mL + a);
        else {
#pragma unroll
          for (int j = 0; j < D::n; ++j) r = fma(T.WL_P[j][b], SM(O::TQ, D::n * D::mm + D::n * D::mL + j * D::mL + a), r);
        }
        LEz[(size_t)k * D::NW + it] += f * r;
      }
    }
  }
  // stage 6: x-pass onto DG nodes, velocity and energy rates, SSP combination
  // (mode 2: the raw Lorentz load C_B^T J, no mass or density division)
  const double tau = MODE == 1 ? dtp[0] * dtfac : 0.0;
  constexpr int I6 = D::n2;
  FLAT(I6) {
    int q = idx / D::EB, e = idx % D::EB, k = k0 + e;
    if (k >= M.K) continue;
    int j = q / D::n, i = q % D::n;
    // second passes: s_x x-pass, s_y y-pass, s_z x-pass of VZ1 and y-pass of HZ
    double sx = 0.0, sy = 0.0, sz = 0.0;
    if constexpr (D::LID) {
      sx = SM(O::VX, j * D::mL + i);
      sy = SM(O::HY, j * D::n + i);
    } else {
#pragma unroll
      for (int a = 0; a < D::mL; ++a) {
        sx = fma(T.P_L[a][i], SM(O::VX, j * D::mL + a), sx);
        sy = fma(T.P_L[a][j], SM(O::HY, a * D::n + i), sy);
      }
    }
    if constexpr (!R2) {
#pragma unroll
      for (int a = 0; a < D::mm; ++a) {
        sz = fma(T.P_G[a][i], SM(O::VZ1, j * D::mm + a), sz);
        sz = fma(T.P_G[a][j], SM(O::HZ, a * D::n + i), sz);
      }
    }
    size_t gq = MHD_CHK((size_t)k * D::n2 + q, N);
    if (MODE == 2) {
      uo[gq] = sx;
      uo[N + gq] = sy;
      uo[2 * N + gq] = sz;
      continue;
    }
    double r_ = rho[gq];
    double im = rcp(r_ * sMW[q]);
    double du[3] = {sx * im, sy * im, sz * im};
    double de = 0.0;
    const double et = SM(O::ETA, 0);
    if (resistive && et != 0.0) {
      double jx = R2 ? 0.0 : SM(O::JQ, q), jy = R2 ? 0.0 : SM(O::JQ, D::n2 + q), jz = SM(O::JQ, 2 * D::n2 + q);
      de = et * fma(jx, jx, fma(jy, jy, jz * jz)) * rcp(r_);
    }
    if (MODE == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) uo[d * N + gq] = du[d];
      eo[gq] = de;
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double raw = fma(tau, du[d], u[d * N + gq]);
        uo[d * N + gq] = first ? raw : fma(ca, u0[d * N + gq], cb * raw);
      }
      double raw = fma(tau, de, e_in[gq]);
      eo[gq] = first ? raw : fma(ca, e0[gq], cb * raw);
    }
  }
}

// ============================ k_mag_B ==========================================
template <int P, int KM>
struct LB_ {
  using D = MD<P, KM>;
  static constexpr int EX = 0, EY = EX + D::NX, EZ = EY + D::NY;
  static constexpr int TY = EZ + D::NW;          // d/dx of E_y rows at GLL(k) x: [b < mm][a < mm]
  static constexpr int TX = TY + D::NZ;          // E_x rows (GLL y) to GLL(k) x: [b < mL][a < mm]
  // per-block assembly factors (closure_factors: NX + NY + NW doubles), at least 8 elements per block
  static constexpr int FAC = TX + D::mL * D::mm;
  static constexpr int SIZE = FAC + (D::NX + D::NY + D::NW + 7) / 8;
};

// mode 0: write dB; mode 1: SSP combination into Bo.
template <int P, int KM, int MODE, int EBv = mag_tile_eb(0), bool R2 = false>
__global__ void __launch_bounds__(256) k_mag_B(const double* __restrict__ LEx, const double* __restrict__ LEy,
                                               const double* __restrict__ LEz, const double* B, const double* B0,
                                               double* Bo, Mesh M, const double* __restrict__ dtp, double dtfac,
                                               double ca, double cb, int first) {
  using D = MD<P, KM, EBv>;
  using O = LB_<P, KM>;
  const MTab& T = c_mtab[D::SLOT];
  extern __shared__ double sm[];
  const int k0 = blockIdx.x * D::EB;
  const size_t Z = (size_t)M.K * D::NZ;
  static_assert(D::EB >= 8, "per-block factor slots assume at least 8 elements per block");
  double* const sAF = sm + (size_t)O::FAC * D::EB;  // assembly factors [NX | NY | NW]
  closure_factors<P, KM>(sAF, nullptr, M);
  __syncthreads();
  // 2D2V (R2): E_x = E_y = 0, so only E_z is assembled and dB_z = 0
  constexpr int I1 = (R2 ? 0 : D::NX + D::NY) + D::NW;
  FLAT(I1) {
    int it = idx / D::EB, e = idx % D::EB, k = min(k0 + e, M.K - 1);
    int ex = k % M.nx, ey = k / M.nx;
    if constexpr (R2) it += D::NX + D::NY;
    const double f = sAF[it];
    if (it < D::NX) SM(O::EX, it) = assemble_Nx_sum<P, KM>(LEx, ex, ey, it % D::mm, it / D::mm, M) * f;
    else if (it < D::NX + D::NY) { it -= D::NX; SM(O::EY, it) = assemble_Ny_sum<P, KM>(LEy, ex, ey, it % D::mL, it / D::mL, M) * f; }
    else { it -= D::NX + D::NY; SM(O::EZ, it) = assemble_W_sum<P, KM>(LEz, ex, ey, it % D::mL, it / D::mL, M) * f; }
  }
  __syncthreads();
  constexpr int I2 = R2 ? 0 : D::NZ + D::mL * D::mm;
  FLAT(I2) {
    int it = idx / D::EB, e = idx % D::EB;
    if (it < D::NZ) {  // d/dx E_y at GLL(k) x, rows Gauss y
      int b = it / D::mm, a = it % D::mm;
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mL; ++c) v = fma(T.dL_M[a][c], SM(O::EY, b * D::mL + c), v);
      SM(O::TY, it) = v;
    } else {
      it -= D::NZ;
      int b = it / D::mm, a = it % D::mm;  // E_x rows (GLL y) to GLL(k) x
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) v = fma(T.G_M[a][c], SM(O::EX, b * D::mm + c), v);
      SM(O::TX, it) = v;
    }
  }
  __syncthreads();
  const double tau = MODE ? dtp[0] * dtfac : 0.0;
  const double ax = 2.0 * M.ihx, ay = 2.0 * M.ihy;
  constexpr int I3 = 3 * D::NZ;
  FLAT(I3) {
    int it = idx / D::EB, e = idx % D::EB, k = k0 + e;
    if (k >= M.K) continue;
    int comp = it / D::NZ, r = it % D::NZ, b = r / D::mm, a = r % D::mm;
    double dB;
    if (comp == 0) {  // Bx at (xL_a, zG_b): -d_y E_z
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mL; ++c) v = fma(T.dL_G[b][c], SM(O::EZ, c * D::mL + a), v);
      dB = -ay * v;
    } else if (comp == 1) {  // By at (zG_a, xL_b): d_x E_z
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < D::mL; ++c) v = fma(T.dL_G[a][c], SM(O::EZ, b * D::mL + c), v);
      dB = ax * v;
    } else if (R2) {
      dB = 0.0;
    } else {  // Bz at (xM_a, xM_b): -(d_x E_y - d_y E_x)
      double vy = 0.0, vx = 0.0;
#pragma unroll
      for (int c = 0; c < D::mm; ++c) vy = fma(T.G_M[b][c], SM(O::TY, c * D::mm + a), vy);
#pragma unroll
      for (int c = 0; c < D::mL; ++c) vx = fma(T.dL_M[b][c], SM(O::TX, c * D::mm + a), vx);
      dB = -fma(ax, vy, -ay * vx);
    }
    size_t gi = MHD_CHK(comp * Z + (size_t)k * D::NZ + r, 3 * Z);
    if (MODE == 0) Bo[gi] = dB;
    else {
      double raw = fma(tau, dB, B[gi]);
      Bo[gi] = first ? raw : fma(ca, B0[gi], cb * raw);
    }
  }
}

// ---- launchers ------------------------------------------------------------------
// Each of the three kernels takes its own tile variant: the mesh's magnetic
// tile code is vE + 3 vJ + 9 vB (a single variant v is v + 3 v + 9 v).
template <int P, int KM, int EBv>
void mag_J_eb(const double* B, double* LJ, const Mesh& M, int reduced, cudaStream_t st) {
  using D = MD<P, KM, EBv>;
  const size_t Z = (size_t)M.K * D::NZ;
  double* LJx = LJ; double* LJy = LJ + (size_t)M.K * D::NX; double* LJz = LJy + (size_t)M.K * D::NY;
  const unsigned blocks = (unsigned)((M.K + D::EB - 1) / D::EB);
  const size_t sj = sizeof(double) * LJ_<P, KM>::SIZE * D::EB;
  if (reduced) k_mag_J<P, KM, EBv, true><<<blocks, D::TH, sj, st>>>(B, B + Z, B + 2 * Z, LJx, LJy, LJz, M);
  else k_mag_J<P, KM, EBv><<<blocks, D::TH, sj, st>>>(B, B + Z, B + 2 * Z, LJx, LJy, LJz, M);
}

template <int P, int KM, int EBv>
void mag_E_eb(int mode, const double* B, const double* u, const double* e, const double* rho, const double* eta,
              int resistive, const double* u0, const double* e0, double* uo, double* eo, const double* LJ, double* LE,
              const Mesh& M, const double* dtp, double dtfac, double ca, double cb, int first, int reduced,
              cudaStream_t st) {
  using D = MD<P, KM, EBv>;
  const size_t Z = (size_t)M.K * D::NZ;
  const double* LJx = LJ; const double* LJy = LJ + (size_t)M.K * D::NX; const double* LJz = LJy + (size_t)M.K * D::NY;
  double* LEx = LE; double* LEy = LE + (size_t)M.K * D::NX; double* LEz = LEy + (size_t)M.K * D::NY;
  const unsigned blocks = (unsigned)((M.K + D::EB - 1) / D::EB);
  const size_t se = sizeof(double) * LE_<P, KM>::SIZE * D::EB;
#define MHD_MAG_E_LAUNCH(MODE_, R2_)                                                                          \
  k_mag_E<P, KM, MODE_, EBv, R2_><<<blocks, D::TH, se, st>>>(LJx, LJy, LJz, B, B + Z, B + 2 * Z, u, e, rho, eta, \
                                                             u0, e0, uo, eo, LEx, LEy, LEz, M, dtp, dtfac, ca, cb, \
                                                             first, resistive)
  if (reduced) {  // 2D2V: u_z = B_z = 0, in-plane E and J vanish
    if (mode == 0) MHD_MAG_E_LAUNCH(0, true);
    else MHD_MAG_E_LAUNCH(1, true);
  } else {
    if (mode == 0) MHD_MAG_E_LAUNCH(0, false);
    else MHD_MAG_E_LAUNCH(1, false);
  }
#undef MHD_MAG_E_LAUNCH
}

template <int P, int KM, int EBv>
void mag_B_eb(int mode, const double* B, const double* B0, double* Bo, const double* LE, const Mesh& M,
              const double* dtp, double dtfac, double ca, double cb, int first, int reduced, cudaStream_t st) {
  using D = MD<P, KM, EBv>;
  const double* LEx = LE; const double* LEy = LE + (size_t)M.K * D::NX; const double* LEz = LEy + (size_t)M.K * D::NY;
  const unsigned blocks = (unsigned)((M.K + D::EB - 1) / D::EB);
  const size_t sb = sizeof(double) * LB_<P, KM>::SIZE * D::EB;
  if (reduced) {
    if (mode == 0) k_mag_B<P, KM, 0, EBv, true><<<blocks, D::TH, sb, st>>>(LEx, LEy, LEz, B, B0, Bo, M, dtp, dtfac, ca, cb, first);
    else k_mag_B<P, KM, 1, EBv, true><<<blocks, D::TH, sb, st>>>(LEx, LEy, LEz, B, B0, Bo, M, dtp, dtfac, ca, cb, first);
  } else {
    if (mode == 0) k_mag_B<P, KM, 0, EBv><<<blocks, D::TH, sb, st>>>(LEx, LEy, LEz, B, B0, Bo, M, dtp, dtfac, ca, cb, first);
    else k_mag_B<P, KM, 1, EBv><<<blocks, D::TH, sb, st>>>(LEx, LEy, LEz, B, B0, Bo, M, dtp, dtfac, ca, cb, first);
  }
}

// Tile variants whose shared memory fits the device (set at context creation).
static bool g_mag_tile_ok[8][kTileVariants] = {};

template <int P, int KM>
void mag_stage_impl(int mode, const double* B, const double* u, const double* e, const double* rho,
                    const double* eta, int resistive, const double* B0, const double* u0, const double* e0,
                    double* Bo, double* uo, double* eo, double* LJ, double* LE, const Mesh& M, const double* dtp,
                    double dtfac, double ca, double cb, int first, int reduced, cudaStream_t st) {
  const int code = M.tile_mag >= 0 && M.tile_mag < kTileVariants * kTileVariants * kTileVariants ? M.tile_mag : 0;
  auto ok = [](int v) { return v > 0 && g_mag_tile_ok[P - 1 + KM][v] ? v : 0; };
  const int vE = ok(code % kTileVariants), vJ = ok(code / kTileVariants % kTileVariants),
            vB = ok(code / (kTileVariants * kTileVariants));
  switch (vJ) {
    case 1: mag_J_eb<P, KM, mag_tile_eb(1)>(B, LJ, M, reduced, st); break;
    case 2: mag_J_eb<P, KM, mag_tile_eb(2)>(B, LJ, M, reduced, st); break;
    default: mag_J_eb<P, KM, mag_tile_eb(0)>(B, LJ, M, reduced, st); break;
  }
#define MHD_MAG_E_EB(V)                                                                                          \
  mag_E_eb<P, KM, mag_tile_eb(V)>(mode, B, u, e, rho, eta, resistive, u0, e0, uo, eo, LJ, LE, M, dtp, dtfac, ca, cb, \
                                  first, reduced, st)
  switch (vE) {
    case 1: MHD_MAG_E_EB(1); break;
    case 2: MHD_MAG_E_EB(2); break;
    default: MHD_MAG_E_EB(0); break;
  }
#undef MHD_MAG_E_EB
#define MHD_MAG_B_EB(V) mag_B_eb<P, KM, mag_tile_eb(V)>(mode, B, B0, Bo, LE, M, dtp, dtfac, ca, cb, first, reduced, st)
  switch (vB) {
    case 1: MHD_MAG_B_EB(1); break;
    case 2: MHD_MAG_B_EB(2); break;
    default: MHD_MAG_B_EB(0); break;
  }
#undef MHD_MAG_B_EB
}

// Opt-in dynamic shared memory of the magnetic kernels of one (p, k) pair on the
// current device (done at context creation, never during stream capture).
template <int P, int KM, int EBv>
static cudaError_t mag_prepare_eb() {
  using D = MD<P, KM, EBv>;
  const int sj = (int)(sizeof(double) * LJ_<P, KM>::SIZE * D::EB);
  const int se = (int)(sizeof(double) * LE_<P, KM>::SIZE * D::EB);
  const int sb = (int)(sizeof(double) * LB_<P, KM>::SIZE * D::EB);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_J<P, KM, EBv>, cudaFuncAttributeMaxDynamicSharedMemorySize, sj);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_E<P, KM, 0, EBv>, cudaFuncAttributeMaxDynamicSharedMemorySize, se);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_E<P, KM, 1, EBv>, cudaFuncAttributeMaxDynamicSharedMemorySize, se);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_B<P, KM, 0, EBv>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_B<P, KM, 1, EBv>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_J<P, KM, EBv, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sj);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_E<P, KM, 0, EBv, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, se);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_E<P, KM, 1, EBv, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, se);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_B<P, KM, 0, EBv, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_mag_B<P, KM, 1, EBv, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
  return e;
}

// The default variant must fit; the others are marked usable when they do.
template <int P, int KM>
static cudaError_t mag_prepare_impl() {
  using D = MD<P, KM>;
  int maxsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t per = sizeof(double) * (size_t)(LE_<P, KM>::SIZE > LJ_<P, KM>::SIZE
                                                    ? (LE_<P, KM>::SIZE > LB_<P, KM>::SIZE ? LE_<P, KM>::SIZE : LB_<P, KM>::SIZE)
                                                    : (LJ_<P, KM>::SIZE > LB_<P, KM>::SIZE ? LJ_<P, KM>::SIZE : LB_<P, KM>::SIZE));
  (void)D::EB;
  cudaError_t e = mag_prepare_eb<P, KM, mag_tile_eb(0)>();
  if (e != cudaSuccess) return e;
  g_mag_tile_ok[P - 1 + KM][0] = true;
  if (per * mag_tile_eb(1) <= (size_t)maxsm && mag_prepare_eb<P, KM, mag_tile_eb(1)>() == cudaSuccess)
    g_mag_tile_ok[P - 1 + KM][1] = true;
  if (per * mag_tile_eb(2) <= (size_t)maxsm && mag_prepare_eb<P, KM, mag_tile_eb(2)>() == cudaSuccess)
    g_mag_tile_ok[P - 1 + KM][2] = true;
  cudaGetLastError();  // a refused opt-in only disables that variant
  return cudaSuccess;
}

cudaError_t mag_prepare(int p, int k) {
  cudaError_t e = cudaErrorInvalidValue;
#define MHD_MAG_PREP(PP, KK) e = mag_prepare_impl<PP, KK>()
  MHD_DISPATCH_PK(p, k, MHD_MAG_PREP);
#undef MHD_MAG_PREP
  return e;
}

#include "magnetic_adjoint.inc"

// Whether tile variant v of the magnetic kernels is usable for (p, k) on this device.
bool mag_tile_ok(int p, int k, int v) {
  const int slot = table_slot(p, k);
  return slot >= 0 && v >= 0 && v < kTileVariants && g_mag_tile_ok[slot][v];
}

size_t mag_load_doubles(int p, int k, int K) {
  (void)p;
  int mm = k + 1, mL = k + 2;
  return (size_t)K * (2 * mm * mL + mL * mL);
}

void mag_stage(int p, int k, int mode, const double* B, const double* u, const double* e, const double* rho,
               const double* eta, int resistive, const double* B0, const double* u0, const double* e0, double* Bo,
               double* uo, double* eo, double* LJ, double* LE, const Tab* T, const Mesh& M, const double* dtp,
               double dtfac, double ca, double cb, int first, int reduced, cudaStream_t st) {
  (void)T;  // the magnetic kernels read the constant-memory copy of the tables
#define MHD_MAG_CASE(PP, KK)                                                                                  \
  mag_stage_impl<PP, KK>(mode, B, u, e, rho, eta, resistive, B0, u0, e0, Bo, uo, eo, LJ, LE, M, dtp, dtfac, ca, \
                         cb, first, reduced, st)
  MHD_DISPATCH_PK(p, k, MHD_MAG_CASE);
#undef MHD_MAG_CASE
}

MHD_OOB_READER(oob_magnetic)

}  // namespace mhd
