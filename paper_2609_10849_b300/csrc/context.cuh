// Private context of the C ABI (include/mhd.h) shared by the translation units
// that drive kernels: the step driver (api.cu) and the adjoint (adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "mhd_internal.cuh"

namespace mhd {
// Kernel launches of the stabilisation launchers, for the contexts' launch counts:
// the sensor statistics (k_stats, k_lines, k_global) and the A.R. coefficient
// (k_ar_elem, k_ar_part, k_ar_global, k_ar_eta).
constexpr int kStatsLaunches = 3;
constexpr int kArLaunches = 4;
// kernels / launchers defined in the other translation units
void hydro_face(int p, const double* S, double* Fx, double* Fy, const Mesh& M, cudaStream_t st);
void hydro_vol(int p, int mode, const double* S, const double* U0, const double* Fx, const double* Fy, double* out,
               double* avg, unsigned* status, const Tab* T, const Mesh& M, const double* dtp, double dtfac,
               double ca, double cb, int first, cudaStream_t st);
size_t mag_load_doubles(int p, int k, int K);
void mag_stage(int p, int k, int mode, const double* B, const double* u, const double* e, const double* rho,
               const double* eta, int resistive, const double* B0, const double* u0, const double* e0, double* Bo,
               double* uo, double* eo, double* LJ, double* LE, const Tab* T, const Mesh& M, const double* dtp,
               double dtfac, double ca, double cb, int first, int reduced, cudaStream_t st);
void grid_to_blocked(const double* g, double* o, int nx, int ny, int mm, cudaStream_t st);
void check_planar(const double* mz, size_t N, const double* bz, size_t Z, unsigned* status, cudaStream_t st);
void l2_project(int k, int nq, const double* fq, double* out, size_t K, cudaStream_t st);
void blocked_to_grid(const double* o, double* g, int nx, int ny, int mm, cudaStream_t st);
void cons_to_prim(const double* U, double* Y, size_t N, cudaStream_t st);
void prim_to_cons(const double* Y, double* U, size_t N, cudaStream_t st);
void prim_in(const double* rho, const double* u, const double* p, double* U, size_t N, double g, cudaStream_t st);
void prim_in_vjp(const double* rho, const double* u, const double* lam, double* G, size_t N, double ig1,
                 cudaStream_t st);
void b_from_potential(int k, const double* A, double Bx0, double By0, double* Bx, double* By, const Tab* T,
                      const Mesh& M, cudaStream_t st);
void cfl_dt(int p, int k, const double* U, const double* B, const Tab* T, const Mesh& M,
            unsigned long long* maxbits, double cfl, double* dt, cudaStream_t st);
void set_scalar(double* ptr, double v, cudaStream_t st);
void mirror_fill(int p, int k, double* U, double* B, const Mesh& M, int pnx, int pny, int walls, int cond,
                 cudaStream_t st);
void diag_partials(int p, int k, const double* U, const double* B, const Tab* T, const Mesh& M, double* out,
                   cudaStream_t st);
void stab_hydro(int p, double* S, unsigned* status, const Tab* T, const Mesh& M, const Stab& prm, const double* dtp,
                double dtfac, double* work, double* frz, cudaStream_t st);
void stab_hydro_adjoint(int p, double* lam, const double* frz, const Tab* T, const Mesh& M, int oe, int pp,
                        cudaStream_t st);
void stab_eta(int p, int k, const double* rho, const double* Y, const double* B, const Tab* T, const Mesh& M,
              const Stab& prm, double* eta, double* work, cudaStream_t st);
void stab_vel_prep(int p, const double* rho, double* chol, const Tab* T, const Mesh& M, cudaStream_t st);
void stab_vel(int p, int k, const double* rho, double* Y, const double* B, const double* chol, const Tab* T,
              const Mesh& M, const Stab& prm, const double* dtp, double dtfac, double* work, double* frz,
              cudaStream_t st);
void stab_vel_adjoint(int p, const double* rho, double* lam, const double* ustar, const double* chol,
                      const double* frzD, const Tab* T, const Mesh& M, cudaStream_t st);
size_t stab_work_doubles(int p, int k, const Mesh& M);
cudaError_t stab_init_mesh(int p, const Tab& hT, const Mesh& M, double* work);
size_t stab_chol_doubles(int p, const Mesh& M);
void set_error_message(const char* msg);
cudaError_t mag_prepare(int p, int k);
cudaError_t stab_prepare(int p);
// adjoint (adjoint_hydro.cu, magnetic_adjoint.inc)
void hydro_rhs_vjp(int p, const double* S, const double* nu, double* FA, double* out, const Mesh& M, const Tab* T,
                   cudaStream_t st);
void axpby(double a, const double* x, double b, double* y, size_t n, cudaStream_t st);
void adj_prim_to_cons(const double* U, const double* Y, const double* lamU, double* lamY, double* lamR, size_t N,
                      cudaStream_t st);
void adj_cons_to_prim(const double* U, const double* lamY, const double* lamR, double* lamU, size_t N,
                      cudaStream_t st);
cudaError_t mag_adj_prepare(int p, int k);
bool mag_tile_ok(int p, int k, int v);
size_t mag_adj_load_doubles(int p, int k, int K);
void mag_rhs_vjp(int p, int k, const double* rho, const double* u, const double* B, const double* we,
                 const double* wu, const double* wB, const double* eta, double* gu, double* gB, double* grho,
                 double rho_scale, const MagAdjScratch& S, const Mesh& M, cudaStream_t st);
}  // namespace mhd

// Stage states of one recomputed Strang step (the adjoint's tape).
struct StepTape {
  double* hS[2][3] = {};     // stage inputs of the two hydro substeps [5N]
  double* Ua = nullptr;      // state after the first hydro substep [5N]
  double* Y[4] = {};         // magnetic stage states (e [N], u [3N], B [3Z] contiguous)
  double* frz = nullptr;     // frozen stage-map coefficients [2][3][K][p+3]
  double* vfrz = nullptr;    // frozen velocity-OE factors [3][K][p+1]
  double* vstar = nullptr;   // velocity before the velocity OE, per magnetic stage [3][3N]
  double* eta = nullptr;     // frozen A.R. coefficient of the magnetic substep [K]
  double* chol = nullptr;    // velocity-OE projectors of the step [K][(p+1)^4] (velocity OE only)
};

// Device buffers of the adjoint, allocated on the first adjoint call; tapes
// grow to the longest segment requested.
struct AdjBufs {
  bool ready = false;
  std::vector<StepTape> tapes;
  double* lamU = nullptr;  // [5N]
  double* lamM = nullptr;  // magnetic adjoint (e, u, B) [4N + 3Z]
  double* W = nullptr;     // stage adjoint input [max(5N, 4N + 3Z)]
  double* L0 = nullptr;    // accumulated adjoint of the substep input
  double* G = nullptr;     // residual VJP; also the scratch end state of a recomputed step
  double* lamR = nullptr;  // adjoint of the frozen density [N]
  double* FA = nullptr;    // face adjoints [2][2][5][K (p+1)]
  double* io = nullptr;    // packed host-layout staging [5N + 3Z]
  mhd::MagAdjScratch ms{};
};

struct mhd_ctx {
  int p, k, n, n2, mm;
  mhd::Mesh M;
  mhd::Stab prm;
  double x0, x1, y0, y1;
  cudaStream_t st;
  bool own_stream;
  const mhd::Tab* T;
  mhd::Tab hT;
  size_t N, Z;
  double *U, *Usave, *S1, *S2;
  double *B, *Bsave, *Ba, *Bb;
  double *Y0, *Ya, *Yb;
  double *Fx, *Fy, *LJ, *LE, *eta, *dt, *work, *chol, *io;
  unsigned* status;
  unsigned long long* maxbits;
  double* h_pinned;  // small pinned host scratch
  unsigned* h_status;
  long long launches;
  long long rejections;  // rejected step attempts since creation
  std::vector<void*> allocs;
  // optional per-kernel-class event timing (bench instrumentation)
  bool profiling;
  // cached CUDA graph of a fixed-dt sequence of Strang steps (mhd_strang_steps)
  cudaGraphExec_t graph;
  int graph_steps;
  long long graph_launches;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_rec;
  AdjBufs adj;
  // reflecting walls by the method of images (mhd_create_walled): bit 0 x, bit 1 y;
  // the physical elements are ex < pnx, ey < pny of the doubled periodic mesh
  int walls, cond, pnx, pny;
};
