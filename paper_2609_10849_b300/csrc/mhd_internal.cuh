// Internal declarations of the B300 H-M-H Strang-step library.
//
// Device layouts (element-blocked; the host layouts of include/mhd.h are
// converted on the way in and out):
//   DG fields          [c][K][n2], n = p+1, node j*n+i           (as on the host)
//   magnetic arrays    [K][mm*mm], mm = k+1, local index b*mm+a   (owned DOFs):
//     Bx  (R, x-comp)  a = GLL(k+1) node 0..k in x, b = Gauss(k) node in y
//     By  (R, y-comp)  a = Gauss(k) node in x,     b = GLL(k+1) node 0..k in y
//     Bz  (V_h^k)      GLL(k) nodes
//   element closures   an element also uses the a = k+1 column / b = k+1 row
//                      of its +x / +y neighbour (node 0 there).
//   per-element loads  closure-sized scratch written by one kernel and
//                      gathered (assembled) by the next.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MHD_NMAX 5  // p + 1 <= 5 and k + 1 <= 5
#define MHD_LMAX 6  // k + 2 <= 6
#define MHD_QMAX 16  // points per direction of element data given at Gauss points

namespace mhd {

// 1D tables of one (p, k) pair.  Row index first: T[a][c] = basis c at point a.
struct Tab {
  double xp[MHD_NMAX], wp[MHD_NMAX];          // GLL(p)
  double D[MHD_NMAX][MHD_NMAX];               // D[i][j] = l_j'(xp_i)
  double xL[MHD_LMAX], wL[MHD_LMAX];          // GLL(k+1)
  double zG[MHD_NMAX], wG[MHD_NMAX];          // Gauss(k), k+1 points
  double xM[MHD_NMAX], wM[MHD_NMAX];          // GLL(k)
  double ML[MHD_LMAX][MHD_LMAX];              // exact GLL(k+1) mass  int l_a l_b
  double dL_G[MHD_NMAX][MHD_LMAX];            // l^L_c'(zG_a)
  double L_G[MHD_NMAX][MHD_LMAX];             // l^L_c(zG_a)
  double G_L[MHD_LMAX][MHD_NMAX];             // g_c(xL_a)
  double M_G[MHD_NMAX][MHD_NMAX];             // l^M_c(zG_a)
  double M_L[MHD_LMAX][MHD_NMAX];             // l^M_c(xL_a)
  double P_G[MHD_NMAX][MHD_NMAX];             // l^P_c(zG_a)
  double P_L[MHD_LMAX][MHD_NMAX];             // l^P_c(xL_a)
  double dL_M[MHD_NMAX][MHD_LMAX];            // l^L_c'(xM_a)
  double G_M[MHD_NMAX][MHD_NMAX];             // g_c(xM_a)
  double L_P[MHD_NMAX][MHD_LMAX];             // l^L_c(xp_a)
  double G_P[MHD_NMAX][MHD_NMAX];             // g_c(xp_a)
  double M_P[MHD_NMAX][MHD_NMAX];             // l^M_c(xp_a)
  double dL_L[MHD_LMAX][MHD_LMAX];            // l^L_c'(xL_a)
  double dL_Gz[MHD_NMAX][MHD_LMAX];           // same as dL_G (kept for symmetry of use)
  double Dr0[MHD_NMAX][MHD_NMAX];             // row 0 of D^r: [r][s]
  double Drp[MHD_NMAX][MHD_NMAX];             // row p of D^r: [r][s]
  double Leg[MHD_NMAX][MHD_NMAX];             // Legendre P_a(xp_i): [i][a]
  double LegN[MHD_NMAX];                      // 1 / sum_i wp_i P_a(xp_i)^2
  double z2[MHD_LMAX], w2[MHD_LMAX];          // Gauss with k+2 points
  double L_2[MHD_LMAX][MHD_LMAX];             // l^L_c(z2_a)
  double G_2[MHD_LMAX][MHD_NMAX];             // g_c(z2_a)
  double M_2[MHD_LMAX][MHD_NMAX];             // l^M_c(z2_a)
  double L_end[2][MHD_LMAX];                  // l^L_c(-1), l^L_c(+1)
  double G_end[2][MHD_NMAX];                  // g_c(-1), g_c(+1)
  double M_end[2][MHD_NMAX];                  // l^M_c(-1), l^M_c(+1)
  double WG_P[MHD_NMAX][MHD_NMAX];            // wp_a g_c(xp_a)
  double WL_P[MHD_NMAX][MHD_LMAX];            // wp_a l^L_c(xp_a)
  double iwLs[MHD_LMAX];                      // 1 / assembled GLL(k+1) weight (2 wL_0 at a = 0)
  double iwG[MHD_NMAX];                       // 1 / wG
  double Wq[MHD_NMAX * MHD_NMAX];             // 0.25 wp_i wp_j at node j*(p+1)+i (element-average weights)
  double hwp[MHD_NMAX];                       // 0.5 wp_i
  // products of two entries that inner loops would otherwise form per iteration
  double WLeg[MHD_NMAX][MHD_NMAX];            // wp_j P_b(xp_j): [j][b]
  double LegLeg[MHD_NMAX][MHD_NMAX][MHD_NMAX];  // P_b(xp_j) P_b2(xp_j): [j][b][b2]
  // the modal basis at the nodes, P_a(xp_i) P_b(xp_j) at node q = j (p+1) + i, basis
  // index alpha in shell order (shell l = max(a, b) holds alpha in [l^2, (l+1)^2))
  double Phi[MHD_NMAX * MHD_NMAX][MHD_NMAX * MHD_NMAX];
  // the x-direction filter of y-mode b of the hydro OE map (sum-factorised):
  // K_b[i][i'] = sum_a D_max(a,b) N_b R_a[i][i'], R_a[i][i'] = N_a P_a(xp_i) wp_i' P_a(xp_i'),
  // split as D_b OES[b] + sum_{a > b} D_a OEQ[b][a] (host sums in long double, rounded once)
  double OES[MHD_NMAX][MHD_NMAX][MHD_NMAX];              // [b][i][i'] = N_b sum_{a <= b} R_a[i][i']
  double OEQ[MHD_NMAX][MHD_NMAX][MHD_NMAX][MHD_NMAX];    // [b][a][i][i'] = N_b R_a[i][i']
};

// Device copy of the tables of the 8 supported (p, k) pairs.
int table_slot(int p, int k);
const Tab* device_tables(int p, int k, cudaError_t* err);  // uploads once per device
void host_tables(int p, int k, Tab* out);
void gauss_points(int nq, double* z);
void l2_projection_table(int k, int nq, double* P);

struct Mesh {
  int nx, ny, K;
  double hx, hy, Jdet, g;
  // tile variants chosen by the autotuner (0 = default elements per CTA):
  // volume kernel and magnetic-stage kernels
  int tile_vol, tile_mag;
  // reciprocals the kernels use, rounded once on the host (mesh_reciprocals)
  double ihx, ihy, iJ, ig1;
};

// Fill the reciprocal fields of a mesh whose hx, hy, Jdet and g are set.
inline void mesh_reciprocals(Mesh& M) {
  M.ihx = 1.0 / M.hx;
  M.ihy = 1.0 / M.hy;
  M.iJ = 1.0 / M.Jdet;
  M.ig1 = 1.0 / (M.g - 1.0);
}

// Elements per CTA of the tile variants (index 0 is the default).
constexpr int vol_tile_eb(int p, int v) {
  return p == 1 ? (v == 0 ? 32 : v == 1 ? 16 : 64)
       : p == 2 ? (v == 0 ? 32 : v == 1 ? 16 : 8)
       : p == 3 ? (v == 0 ? 8 : v == 1 ? 4 : 16)
                : (v == 0 ? 5 : v == 1 ? 3 : 8);
}
constexpr int mag_tile_eb(int v) { return v == 0 ? 16 : v == 1 ? 8 : 32; }
constexpr int kTileVariants = 3;

// Stabilisation parameters as seen by the kernels.
struct Stab {
  int oe_hydro, oe_vel, pp, ar;
  double s_H, s_M, C_s, C_eta, cfl;
  int max_halvings;
  unsigned* activity;  // device word: which maps acted (ACT_* bits), may be null
  int strang_order;    // 0: H-M-H (Algorithm 3), 1: M-H-M
  int reduced;         // 1: 2D2V magnetic stage (u_z = B_z = 0; in-plane E and J not formed)
};

// Activity bits of the stabilisation maps (mhd_diag_t.stab_active).
enum : unsigned {
  ACT_OE_HYDRO = 1u,  // a hydro OE factor D_p below 0.99
  ACT_PP = 2u,        // the limiter scaled or collapsed an element
  ACT_AR = 4u,        // a positive A.R. coefficient
  ACT_OE_VEL = 8u,    // a velocity-OE factor D_p below 0.99
};

// OR `bits` of the calling lanes of a warp into *word with one atomic per warp.
__device__ __forceinline__ void warp_or(unsigned* word, unsigned bits) {
  const unsigned m = __activemask();
  const unsigned all = __reduce_or_sync(m, bits);
  if (word && all && (threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicOr(word, all);
}

// Scratch of the magnetic-residual adjoint (doubles): mu, s [3N]; LT, LJ, LE
// [element loads of the magnetic stage]; V [3Z]; LB [closure loads of B].
struct MagAdjScratch {
  double *mu, *s, *LT, *LJ, *LE, *V, *LB;
};

// Status word bits written by kernels.
enum : unsigned {
  ST_INADMISSIBLE = 1u,
  ST_NONFINITE = 2u,
  ST_TIMEOUT = 4u,
  ST_NOT_PLANAR = 8u,  // reduced 2D2V stage on a state with u_z or B_z nonzero
};

// ---- debug index checks ---------------------------------------------------------
// Built with -DMHD_BOUNDS_CHECK (libmhd_debug.so), MHD_CHK(i, n) counts every
// index outside [0, n) in a device word of the translation unit and returns 0
// instead, so a bad index is recorded and never dereferenced; the release build
// compiles it to the index itself.  mhd_debug_oob() sums the words.
#ifdef MHD_BOUNDS_CHECK
static __device__ unsigned long long g_oob_count;
__device__ __forceinline__ size_t chk_index(long long i, long long n) {
  if (i < 0 || i >= n) {
    atomicAdd(&g_oob_count, 1ull);
    return 0;
  }
  return (size_t)i;
}
#define MHD_CHK(i, n) (::mhd::chk_index((long long)(i), (long long)(n)))
#define MHD_OOB_READER(name)                                                   \
  unsigned long long name(bool reset) {                                        \
    unsigned long long v = 0;                                                  \
    cudaMemcpyFromSymbol(&v, g_oob_count, sizeof v);                           \
    if (reset) {                                                               \
      const unsigned long long z = 0;                                          \
      cudaMemcpyToSymbol(g_oob_count, &z, sizeof z);                           \
    }                                                                          \
    return v;                                                                  \
  }
#else
#define MHD_CHK(i, n) ((void)sizeof(n), (i))  // n is not evaluated
#define MHD_OOB_READER(name) \
  unsigned long long name(bool) { return 0; }
#endif

__host__ __device__ inline int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---- fast FP64 reciprocal ---------------------------------------------------
// Seed from the documented PTX approximation rcp.approx.ftz.f64 (high-word
// reciprocal, relative error below 2^-22), refined by one cubic Newton-Raphson
// step r1 = r0 (1 + e + e^2), e = 1 - x r0 (error e^3 < 2^-66, then rounding).
// Valid for normal x with |x| in [2^-1000, 2^1000]; the library only takes
// reciprocals of densities, pressures and sums of those.
__device__ __forceinline__ double rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  double t = fma(e, e, e);
  return fma(r, t, r);
}

// ---- fast FP64 square root ----------------------------------------------------
// Heron's (Newton's) iteration for the root, s <- s + (x - s^2) / (2 s), with the
// reciprocal 1/(2 s) taken from the documented PTX seed rsqrt.approx.ftz.f64,
// y ~ x^-1/2 with relative error e << 2^-20, and never refined:
//   s0 = x y = sqrt(x)(1 + e),  s1 = s0 + (x - s0^2) y/2 = sqrt(x)(1 - e^2),
//   s2 = s1 + (x - s1^2) y/2 = sqrt(x)(1 + e^3)  (then one rounding).
// The residuals are single FMAs.  Zero returns itself; subnormal, infinite and
// NaN inputs (which the flushing seed does not cover) take IEEE sqrt; a
// negative normal input gives NaN, as sqrt does.
__device__ __forceinline__ double fsqrt(double x) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
  if (a - 0x0010000000000000ULL >= 0x7fe0000000000000ULL) return a == 0 ? x : sqrt(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = 0.5 * y;
  const double s0 = x * y;
  const double s1 = fma(fma(-s0, s0, x), h, s0);
  return fma(fma(-s1, s1, x), h, s1);
}

// ---- order-preserving integer keys of doubles ---------------------------------
// key(a) < key(b) <=> a < b for non-NaN doubles (-0 sorts below +0), so
// minima and maxima can be taken with 64-bit integer operations, which run on
// the integer pipe instead of the FP64 pipe; dkey_inv(dkey(x)) == x bitwise.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dkey_inv(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// ---- launch counting ----------------------------------------------------------
struct Ctx;
void count_launch(Ctx* c);

}  // namespace mhd

// Dispatch a templated functor over the supported (p, k) pairs.
#define MHD_DISPATCH_PK(p, k, F)                                 \
  do {                                                           \
    switch ((p) * 10 + (k)) {                                    \
      case 10: F(1, 0); break;                                   \
      case 11: F(1, 1); break;                                   \
      case 21: F(2, 1); break;                                   \
      case 22: F(2, 2); break;                                   \
      case 32: F(3, 2); break;                                   \
      case 33: F(3, 3); break;                                   \
      case 43: F(4, 3); break;                                   \
      case 44: F(4, 4); break;                                   \
      default: break;                                            \
    }                                                            \
  } while (0)
