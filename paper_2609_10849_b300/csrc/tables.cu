// One-dimensional rules and interpolation tables of the library (§3.1.3).
//
// Gauss-Legendre and Gauss-Lobatto-Legendre rules are computed in long double
// by Newton's method on the Legendre recurrence; Lagrange bases are evaluated
// in barycentric form (Berrut & Trefethen 2004), derivatives through the
// barycentric differentiation matrix.  Everything is computed once per (p, k)
// pair on the host and uploaded to a device table per device.
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "mhd_internal.cuh"

namespace mhd {
namespace {

typedef long double ld;
const ld PI_L = 3.141592653589793238462643383279502884L;

// P_n(x) and P_n'(x) by the three-term recurrence in long double.
void leg_ld(int n, ld x, ld* P, ld* dP) {
  ld pm1 = 0.0L, p0 = 1.0L;  // P_{-1} = 0 convention keeps the loop uniform
  for (int k = 1; k <= n; ++k) {
    ld pk = ((2 * k - 1) * x * p0 - (k - 1) * pm1) / k;
    pm1 = p0;
    p0 = pk;
  }
  *P = p0;
  // (1 - x^2) P_n' = n (P_{n-1} - x P_n), valid away from the endpoints
  if (n == 0) *dP = 0.0L;
  else *dP = n * (pm1 - x * p0) / (1.0L - x * x);
}

// npts-point Gauss rule on [-1, 1], ascending.
void gauss_ld(int npts, ld* x, ld* w) {
  for (int i = 0; i < npts; ++i) {
    ld z = cosl(PI_L * (4 * i + 3) / (4 * npts + 2));  // i-th root from the right
    for (int it = 0; it < 60; ++it) {
      ld P, dP;
      leg_ld(npts, z, &P, &dP);
      ld dz = P / dP;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    ld P, dP;
    leg_ld(npts, z, &P, &dP);
    x[npts - 1 - i] = z;
    w[npts - 1 - i] = 2.0L / ((1.0L - z * z) * dP * dP);
  }
  for (int i = 0; i < npts / 2; ++i) {  // enforce exact symmetry
    ld a = 0.5L * (x[npts - 1 - i] - x[i]);
    x[i] = -a; x[npts - 1 - i] = a;
    ld b = 0.5L * (w[i] + w[npts - 1 - i]);
    w[i] = b; w[npts - 1 - i] = b;
  }
  if (npts % 2) x[npts / 2] = 0.0L;
}

// GLL rule of degree r (r+1 points): interior nodes are the roots of P_r',
// i.e. of (1-x^2) P_r'; weights 2 / (r (r+1) P_r^2).
void gll_ld(int r, ld* x, ld* w) {
  if (r == 0) { x[0] = 0.0L; w[0] = 2.0L; return; }
  x[0] = -1.0L; x[r] = 1.0L;
  for (int i = 1; i < r; ++i) {
    ld z = -cosl(PI_L * i / r);
    for (int it = 0; it < 60; ++it) {
      // q(z) = P_{r-1}(z) - z P_r(z) = (1-z^2) P_r'(z)/r ; q'(z) = -r(r+1)/r * P_r ... use derivative of q
      ld P, dP;
      leg_ld(r, z, &P, &dP);
      // Newton on P_r' with P_r'' from Legendre's equation
      ld d2P = (2.0L * z * dP - r * (r + 1.0L) * P) / (1.0L - z * z);
      ld dz = dP / d2P;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    x[i] = z;
  }
  for (int i = 0; i <= r; ++i) {
    ld P, dP;
    leg_ld(r, x[i], &P, &dP);
    w[i] = 2.0L / (r * (r + 1.0L) * P * P);
  }
  for (int i = 0; i < (r + 1) / 2; ++i) {
    ld a = 0.5L * (x[r - i] - x[i]);
    x[i] = -a; x[r - i] = a;
    ld b = 0.5L * (w[i] + w[r - i]);
    w[i] = b; w[r - i] = b;
  }
  if (r % 2 == 0) x[r / 2] = 0.0L;
}

// Barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k).
void bary_weights(int n, const ld* xs, ld* lam) {
  for (int j = 0; j < n; ++j) {
    ld p = 1.0L;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (xs[j] - xs[k]);
    lam[j] = 1.0L / p;
  }
}

// Values l_j(x) of all n Lagrange basis functions (first barycentric form).
void lagrange_values(int n, const ld* xs, ld x, ld* v) {
  ld lam[MHD_LMAX + 2];
  bary_weights(n, xs, lam);
  for (int j = 0; j < n; ++j)
    if (x == xs[j]) {
      for (int k = 0; k < n; ++k) v[k] = (k == j) ? 1.0L : 0.0L;
      return;
    }
  ld ell = 1.0L;
  for (int k = 0; k < n; ++k) ell *= (x - xs[k]);
  for (int j = 0; j < n; ++j) v[j] = ell * lam[j] / (x - xs[j]);
}

// Derivatives l_j'(x): l_j' is of degree n-2, so l_j'(x) = sum_i l_i(x) D_ij
// with the barycentric differentiation matrix D_ij = (lam_j/lam_i)/(x_i - x_j).
void lagrange_derivs(int n, const ld* xs, ld x, ld* d) {
  ld lam[MHD_LMAX + 2], Dm[MHD_LMAX + 2][MHD_LMAX + 2], v[MHD_LMAX + 2];
  bary_weights(n, xs, lam);
  for (int i = 0; i < n; ++i) {
    ld s = 0.0L;
    for (int j = 0; j < n; ++j)
      if (j != i) { Dm[i][j] = (lam[j] / lam[i]) / (xs[i] - xs[j]); s += Dm[i][j]; }
    Dm[i][i] = -s;
  }
  lagrange_values(n, xs, x, v);
  for (int j = 0; j < n; ++j) {
    ld s = 0.0L;
    for (int i = 0; i < n; ++i) s += v[i] * Dm[i][j];
    d[j] = s;
  }
}

template <int R, int C>
void fill_interp(double (&T)[R][C], int npts, const ld* pts, int nb, const ld* nodes, bool deriv) {
  for (int a = 0; a < R; ++a)
    for (int c = 0; c < C; ++c) T[a][c] = 0.0;
  for (int a = 0; a < npts; ++a) {
    ld v[MHD_LMAX + 2];
    if (deriv) lagrange_derivs(nb, nodes, pts[a], v);
    else lagrange_values(nb, nodes, pts[a], v);
    for (int c = 0; c < nb; ++c) T[a][c] = (double)v[c];
  }
}

}  // namespace

void gauss_points(int nq, double* z) {
  ld x[MHD_QMAX], w[MHD_QMAX];
  gauss_ld(nq, x, w);
  for (int i = 0; i < nq; ++i) z[i] = (double)x[i];
}

// One-dimensional factor of the L2(K) projection onto Q^k (GLL(k) nodal basis)
// from values at the nq-point Gauss rule: P = M^{-1} L^T W with
// L[g][a] = l_a(zeta_g), W = diag(varpi_g) and M = L^T W L, exact for
// nq >= k + 1.  On a rectangle the element projection of data F[qy][qx] is
// C = P F P^T (the Jacobian cancels).  P is row-major [k+1][nq].
void l2_projection_table(int k, int nq, double* P) {
  const int mm = k + 1;
  ld zq[MHD_QMAX], wq[MHD_QMAX], xM[MHD_NMAX], wM[MHD_NMAX], L[MHD_QMAX][MHD_LMAX + 2];
  gauss_ld(nq, zq, wq);
  gll_ld(k, xM, wM);
  for (int g = 0; g < nq; ++g) lagrange_values(mm, xM, zq[g], L[g]);
  ld A[MHD_NMAX][2 * MHD_NMAX];  // [M | I] -> [I | M^{-1}] by Gauss-Jordan
  for (int a = 0; a < mm; ++a)
    for (int b = 0; b < mm; ++b) {
      ld s = 0.0L;
      for (int g = 0; g < nq; ++g) s += wq[g] * L[g][a] * L[g][b];
      A[a][b] = s;
      A[a][mm + b] = (a == b) ? 1.0L : 0.0L;
    }
  for (int c = 0; c < mm; ++c) {  // M is symmetric positive definite: no pivoting
    ld d = A[c][c];
    for (int j = 0; j < 2 * mm; ++j) A[c][j] /= d;
    for (int r = 0; r < mm; ++r)
      if (r != c) {
        ld f = A[r][c];
        for (int j = 0; j < 2 * mm; ++j) A[r][j] -= f * A[c][j];
      }
  }
  for (int a = 0; a < mm; ++a)
    for (int g = 0; g < nq; ++g) {
      ld s = 0.0L;
      for (int b = 0; b < mm; ++b) s += A[a][mm + b] * L[g][b];
      P[a * nq + g] = (double)(s * wq[g]);
    }
}

void host_tables(int p, int k, Tab* T) {
  std::memset(T, 0, sizeof(Tab));
  const int n = p + 1, mm = k + 1, mL = k + 2;
  ld xp[MHD_NMAX], wp[MHD_NMAX], xL[MHD_LMAX], wL[MHD_LMAX], zG[MHD_NMAX], wG[MHD_NMAX], xM[MHD_NMAX],
      wM[MHD_NMAX], z2[MHD_LMAX], w2[MHD_LMAX];
  gll_ld(p, xp, wp);
  gll_ld(k + 1, xL, wL);
  gll_ld(k, xM, wM);
  gauss_ld(k + 1, zG, wG);
  gauss_ld(k + 2, z2, w2);
  for (int i = 0; i < n; ++i) { T->xp[i] = (double)xp[i]; T->wp[i] = (double)wp[i]; }
  for (int i = 0; i < mL; ++i) { T->xL[i] = (double)xL[i]; T->wL[i] = (double)wL[i]; }
  for (int i = 0; i < mm; ++i) {
    T->zG[i] = (double)zG[i]; T->wG[i] = (double)wG[i];
    T->xM[i] = (double)xM[i]; T->wM[i] = (double)wM[i];
  }
  for (int i = 0; i < k + 2; ++i) { T->z2[i] = (double)z2[i]; T->w2[i] = (double)w2[i]; }
  fill_interp(T->D, n, xp, n, xp, true);
  fill_interp(T->dL_G, mm, zG, mL, xL, true);
  fill_interp(T->dL_Gz, mm, zG, mL, xL, true);
  fill_interp(T->L_G, mm, zG, mL, xL, false);
  fill_interp(T->G_L, mL, xL, mm, zG, false);
  fill_interp(T->M_G, mm, zG, mm, xM, false);
  fill_interp(T->M_L, mL, xL, mm, xM, false);
  fill_interp(T->P_G, mm, zG, n, xp, false);
  fill_interp(T->P_L, mL, xL, n, xp, false);
  fill_interp(T->dL_M, mm, xM, mL, xL, true);
  fill_interp(T->G_M, mm, xM, mm, zG, false);
  fill_interp(T->L_P, n, xp, mL, xL, false);
  fill_interp(T->G_P, n, xp, mm, zG, false);
  fill_interp(T->M_P, n, xp, mm, xM, false);
  fill_interp(T->dL_L, mL, xL, mL, xL, true);
  fill_interp(T->L_2, k + 2, z2, mL, xL, false);
  fill_interp(T->G_2, k + 2, z2, mm, zG, false);
  fill_interp(T->M_2, k + 2, z2, mm, xM, false);
  ld ends[2] = {-1.0L, 1.0L};
  fill_interp(T->L_end, 2, ends, mL, xL, false);
  fill_interp(T->G_end, 2, ends, mm, zG, false);
  fill_interp(T->M_end, 2, ends, mm, xM, false);
  for (int a = 0; a < n; ++a) {
    for (int c = 0; c < mm; ++c) T->WG_P[a][c] = (double)(wp[a] * (ld)T->G_P[a][c]);
    for (int c = 0; c < mL; ++c) T->WL_P[a][c] = (double)(wp[a] * (ld)T->L_P[a][c]);
  }
  for (int a = 0; a < mL; ++a) T->iwLs[a] = (double)(1.0L / (a == 0 ? 2.0L * wL[0] : wL[a]));
  for (int a = 0; a < mm; ++a) T->iwG[a] = (double)(1.0L / wG[a]);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) T->Wq[j * n + i] = 0.25 * T->wp[i] * T->wp[j];
  for (int i = 0; i < n; ++i) T->hwp[i] = 0.5 * T->wp[i];
  // exact GLL(k+1) mass with the (k+2)-point Gauss rule
  for (int a = 0; a < mL; ++a)
    for (int b = 0; b < mL; ++b) {
      ld s = 0.0L;
      for (int q = 0; q < k + 2; ++q) {
        ld v[MHD_LMAX + 2];
        lagrange_values(mL, xL, z2[q], v);
        s += w2[q] * v[a] * v[b];
      }
      T->ML[a][b] = (double)s;
    }
  // rows 0 and p of the powers D^r (r-th derivatives at the element ends)
  ld Dl[MHD_NMAX][MHD_NMAX], Pw[MHD_NMAX][MHD_NMAX], Tm[MHD_NMAX][MHD_NMAX];
  for (int i = 0; i < n; ++i) {
    ld d[MHD_LMAX + 2];
    lagrange_derivs(n, xp, xp[i], d);
    for (int j = 0; j < n; ++j) Dl[i][j] = d[j];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Pw[i][j] = (i == j) ? 1.0L : 0.0L;
  for (int r = 0; r < n; ++r) {
    for (int s = 0; s < n; ++s) { T->Dr0[r][s] = (double)Pw[0][s]; T->Drp[r][s] = (double)Pw[p][s]; }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        ld s = 0.0L;
        for (int q = 0; q < n; ++q) s += Dl[i][q] * Pw[q][j];
        Tm[i][j] = s;
      }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) Pw[i][j] = Tm[i][j];
  }
  // discrete Legendre basis on GLL(p)
  for (int i = 0; i < n; ++i) {
    ld P0 = 1.0L, P1 = xp[i];
    T->Leg[i][0] = 1.0;
    if (n > 1) T->Leg[i][1] = (double)P1;
    for (int a = 2; a < n; ++a) {
      ld P2 = ((2 * a - 1) * xp[i] * P1 - (a - 1) * P0) / a;
      T->Leg[i][a] = (double)P2;
      P0 = P1; P1 = P2;
    }
  }
  for (int a = 0; a < n; ++a) {
    ld s = 0.0L;
    for (int i = 0; i < n; ++i) s += wp[i] * (ld)T->Leg[i][a] * (ld)T->Leg[i][a];
    T->LegN[a] = (double)(1.0L / s);
  }
  // double products exactly as a kernel would form them (one IEEE multiply)
  for (int j = 0; j < n; ++j)
    for (int b = 0; b < n; ++b) {
      T->WLeg[j][b] = T->wp[j] * T->Leg[j][b];
      for (int b2 = 0; b2 < n; ++b2) T->LegLeg[j][b][b2] = T->Leg[j][b] * T->Leg[j][b2];
    }
  {
    int sa[MHD_NMAX * MHD_NMAX], sb[MHD_NMAX * MHD_NMAX], t = 0;
    for (int l = 0; l < n; ++l)
      for (int b = 0; b <= l; ++b)
        for (int a = 0; a <= l; ++a)
          if ((a > b ? a : b) == l) { sa[t] = a; sb[t] = b; ++t; }
    for (int q = 0; q < n * n; ++q)
      for (int al = 0; al < n * n; ++al) T->Phi[q][al] = T->Leg[q % n][sa[al]] * T->Leg[q / n][sb[al]];
  }
  {
    ld Pl[MHD_NMAX][MHD_NMAX], Nl[MHD_NMAX];  // P_a(xp_i) and N_a in long double
    for (int i = 0; i < n; ++i) {
      ld P0 = 1.0L, P1 = xp[i];
      Pl[i][0] = 1.0L;
      if (n > 1) Pl[i][1] = P1;
      for (int a = 2; a < n; ++a) {
        ld P2 = ((2 * a - 1) * xp[i] * P1 - (a - 1) * P0) / a;
        Pl[i][a] = P2;
        P0 = P1; P1 = P2;
      }
    }
    for (int a = 0; a < n; ++a) {
      ld s = 0.0L;
      for (int i = 0; i < n; ++i) s += wp[i] * Pl[i][a] * Pl[i][a];
      Nl[a] = 1.0L / s;
    }
    for (int b = 0; b < n; ++b)
      for (int i = 0; i < n; ++i)
        for (int i2 = 0; i2 < n; ++i2) {
          ld acc = 0.0L;
          for (int a = 0; a < n; ++a) {
            const ld R = Nl[b] * Nl[a] * Pl[i][a] * wp[i2] * Pl[i2][a];
            if (a <= b) acc += R;
            else T->OEQ[b][a][i][i2] = (double)R;
          }
          T->OES[b][i][i2] = (double)acc;
        }
  }
}

int table_slot(int p, int k) {
  switch (p * 10 + k) {
    case 10: return 0; case 11: return 1; case 21: return 2; case 22: return 3;
    case 32: return 4; case 33: return 5; case 43: return 6; case 44: return 7;
    default: return -1;
  }
}

__device__ Tab g_tables[8];
void upload_mag_tables(int slot, const Tab* h, cudaError_t* err);  // constant-memory copy (magnetic.cu)

// Unique id of the current CUDA context (cuCtxGetId, fetched through the
// runtime's driver entry points so the library does not link libcuda), or 0
// where the driver cannot tell.  Keys the upload cache below: a context made
// after cudaDeviceReset() has fresh, empty device symbols and a new id.
static unsigned long long current_context_id() {
  typedef CUresult (*get_current_t)(CUcontext*);
  typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess || q1 != cudaDriverEntryPointSuccess)
      get_current = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess || q2 != cudaDriverEntryPointSuccess)
      get_id = nullptr;
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

const Tab* device_tables(int p, int k, cudaError_t* err) {
  static std::mutex mu;
  static unsigned long long filled_ctx[64][8] = {};  // context id the slot was uploaded in (0: never)
  int slot = table_slot(p, k);
  *err = cudaSuccess;
  if (slot < 0) { *err = cudaErrorInvalidValue; return nullptr; }
  int dev = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) { *err = cudaErrorInvalidDevice; return nullptr; }
  void* base = nullptr;  // also initialises the context, so its id is defined below
  if ((*err = cudaGetSymbolAddress(&base, g_tables)) != cudaSuccess) return nullptr;
  const unsigned long long ctx = current_context_id();
  const unsigned long long key = ctx ? ctx : ~0ull;  // no id: one upload per device
  if (filled_ctx[dev][slot] != key) {
    Tab h;
    host_tables(p, k, &h);
    if ((*err = cudaMemcpyToSymbol(g_tables, &h, sizeof(Tab), slot * sizeof(Tab))) != cudaSuccess) return nullptr;
    upload_mag_tables(slot, &h, err);
    if (*err != cudaSuccess) return nullptr;
    filled_ctx[dev][slot] = key;
  }
  return reinterpret_cast<const Tab*>(base) + slot;
}

}  // namespace mhd
