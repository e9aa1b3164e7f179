// Adjoint of one H-M-H Strang step (Algorithm 3, eq. strang-composition) at
// fixed dt.  The stabilisation maps are differentiated with their
// coefficients frozen at the values of the recomputed forward step: the OE
// factors D_l and limiter factors theta of the hydro stage maps, the factors
// and the rho-weighted projector of the velocity OE, and the A.R. coefficient
// eta (whose resistive Ohm load and Ohmic heating are differentiated).
//
// Reverse mode written out by hand: the step's intermediate states are
// recomputed from its start state (the hydro stage inputs of both hydro
// substeps, the state after the first one and the magnetic stage states),
// then the adjoint runs backwards through
//   Phi_H^{dt/2}  <-  exchange back  <-  Phi_M^{dt}  <-  exchange  <-  Phi_H^{dt/2}.
// Each SSP-RK(3,3) substep (eq. euler-ssprk33, eq. magnetic-ssprk33) is
//   S1 = S0 + tau F(S0),  S2 = 3/4 S0 + 1/4 (S1 + tau F(S1)),
//   S3 = 1/3 S0 + 2/3 (S2 + tau F(S2)),
// whose adjoint for lam3 is, with a = (0, 3/4, 1/3), b = (1, 1/4, 2/3):
//   w = b2 lam3, lam2 = w + tau F'(S2)^T w, lam0  = a2 lam3,
//   w = b1 lam2, lam1 = w + tau F'(S1)^T w, lam0 += a1 lam2,
//   lam0 += lam1 + tau F'(S0)^T lam1.
// The magnetic substep freezes the density, so its adjoint also accumulates
// the density adjoint, which the two exchanges pass on to the conservative
// variables.
#include <algorithm>
#include <string>

#include "../../include/mhd.h"
#include "context.cuh"

using namespace mhd;

namespace {

const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};
const double RK_B[3] = {1.0, 0.25, 2.0 / 3.0};

int afail(int code, const std::string& msg) {
  set_error_message(msg.c_str());
  return code;
}
int acuda(cudaError_t e, const char* where) {
  return afail(MHD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

cudaError_t aalloc(mhd_ctx* c, double** p, size_t n) {
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(n, 1) * sizeof(double));
  if (e == cudaSuccess) { c->allocs.push_back(ptr); *p = (double*)ptr; }
  return e;
}

cudaError_t acopy(mhd_ctx* c, double* dst, const double* src, size_t n, cudaMemcpyKind host_kind, int on_device) {
  return cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : host_kind, c->st);
}

// L0 = a lam (+ L0 if acc), W = b lam.
__global__ void k_lin2(const double* __restrict__ lam, double a, double b, int acc, double* __restrict__ L0,
                       double* __restrict__ W, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l = lam[i];
  L0[i] = acc ? fma(a, l, L0[i]) : a * l;
  W[i] = b * l;
}

// out = W + tau G (acc: out += W + tau G).
__global__ void k_fin(const double* __restrict__ W, const double* __restrict__ G, double tau, int acc,
                      double* __restrict__ out, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = fma(tau, G[i], W[i]);
  out[i] = acc ? out[i] + v : v;
}

unsigned nblk(size_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t alloc_tape(mhd_ctx* c, StepTape& t) {
  const size_t N = c->N, Z = c->Z, K = c->M.K, VM = 4 * N + 3 * Z;
  cudaError_t e = cudaSuccess;
  for (int h = 0; h < 2 && e == cudaSuccess; ++h)
    for (int s = 0; s < 3 && e == cudaSuccess; ++s) e = aalloc(c, &t.hS[h][s], 5 * N);
  if (e == cudaSuccess) e = aalloc(c, &t.Ua, 5 * N);
  for (int s = 0; s < 4 && e == cudaSuccess; ++s) e = aalloc(c, &t.Y[s], VM);
  if (e == cudaSuccess) e = aalloc(c, &t.frz, 6 * K * (c->n + 2));
  if (e == cudaSuccess) e = aalloc(c, &t.vfrz, 3 * K * c->n);
  if (e == cudaSuccess) e = aalloc(c, &t.vstar, 9 * N);
  if (e == cudaSuccess) e = aalloc(c, &t.eta, K);
  return e;
}

int ensure_adjoint(mhd_ctx* c) {
  AdjBufs& A = c->adj;
  if (A.ready) return MHD_OK;
  const size_t N = c->N, Z = c->Z, K = c->M.K;
  const size_t VM = 4 * N + 3 * Z, VX = std::max(5 * N, VM);
  A.tapes.resize(1);
  cudaError_t e = alloc_tape(c, A.tapes[0]);
  if (e == cudaSuccess) e = aalloc(c, &A.lamU, 5 * N);
  if (e == cudaSuccess) e = aalloc(c, &A.lamM, VM);
  if (e == cudaSuccess) e = aalloc(c, &A.W, VX);
  if (e == cudaSuccess) e = aalloc(c, &A.L0, VX);
  if (e == cudaSuccess) e = aalloc(c, &A.G, VX);
  if (e == cudaSuccess) e = aalloc(c, &A.lamR, N);
  if (e == cudaSuccess) e = aalloc(c, &A.FA, 20 * K * c->n);
  if (e == cudaSuccess) e = aalloc(c, &A.io, 5 * N + 3 * Z);
  if (e == cudaSuccess) e = aalloc(c, &A.ms.mu, 3 * N);
  if (e == cudaSuccess) e = aalloc(c, &A.ms.s, 3 * N);
  if (e == cudaSuccess) e = aalloc(c, &A.ms.LT, mag_load_doubles(c->p, c->k, (int)K));
  if (e == cudaSuccess) e = aalloc(c, &A.ms.LJ, mag_load_doubles(c->p, c->k, (int)K));
  if (e == cudaSuccess) e = aalloc(c, &A.ms.LE, mag_load_doubles(c->p, c->k, (int)K));
  if (e == cudaSuccess) e = aalloc(c, &A.ms.V, 3 * Z);
  if (e == cudaSuccess) e = aalloc(c, &A.ms.LB, mag_adj_load_doubles(c->p, c->k, (int)K));
  if (e != cudaSuccess) return afail(MHD_ENOMEM, std::string("adjoint buffers: ") + cudaGetErrorString(e));
  A.ready = true;
  return MHD_OK;
}

// Tapes for m steps (and, with the velocity OE on, their projector storage).
int ensure_tapes(mhd_ctx* c, int m) {
  AdjBufs& A = c->adj;
  cudaError_t e = cudaSuccess;
  while ((int)A.tapes.size() < m && e == cudaSuccess) {
    StepTape t;
    e = alloc_tape(c, t);  // buffers already taken stay owned by the context
    if (e == cudaSuccess) A.tapes.push_back(t);
  }
  if (c->prm.oe_vel)
    for (int i = 0; i < m && e == cudaSuccess; ++i)
      if (!A.tapes[i].chol) e = aalloc(c, &A.tapes[i].chol, stab_chol_doubles(c->p, c->M));
  if (e != cudaSuccess) return afail(MHD_ENOMEM, std::string("adjoint tapes: ") + cudaGetErrorString(e));
  return MHD_OK;
}

// ---- forward recomputation ---------------------------------------------------------
bool stab_on(const mhd_ctx* c) { return c->prm.oe_hydro || c->prm.pp; }
bool resistive(const mhd_ctx* c) { return c->prm.ar && c->prm.C_eta != 0.0; }

double* frz_slot(mhd_ctx* c, StepTape& t, int h, int s) { return t.frz + (size_t)(3 * h + s) * c->M.K * (c->n + 2); }

// Hydro substep h (0 or 1) of tau = dt * fac from S[0] (filled by the caller),
// keeping the stage inputs S[1], S[2] and, with stabilisation on, the frozen
// coefficients of every stage map; the result goes to out.
void hydro_fwd(mhd_ctx* c, StepTape& t, double* out, double fac, int h) {
  double* const* S = t.hS[h];
  const double* in[3] = {S[0], S[1], S[2]};
  double* o[3] = {S[1], S[2], out};
  for (int s = 0; s < 3; ++s) {
    hydro_face(c->p, in[s], c->Fx, c->Fy, c->M, c->st);
    hydro_vol(c->p, 1, in[s], S[0], c->Fx, c->Fy, o[s], nullptr, c->status, c->T, c->M, c->dt, fac, RK_A[s],
              RK_B[s], s == 0, c->st);
    c->launches += 2;
    if (stab_on(c)) {
      stab_hydro(c->p, o[s], c->status, c->T, c->M, c->prm, c->dt, fac, c->work, frz_slot(c, t, h, s), c->st);
      c->launches += c->prm.oe_hydro ? kStatsLaunches + 1 : 1;
    }
  }
}

// Magnetic substep tau = dt * fac from Y[0] (e, u, B) with density rho,
// keeping the stage states Y[1], Y[2]; the result goes to Y[3].  The frozen
// coefficients of the A.R. and of the velocity OE (with the velocity of every
// stage candidate before the filter) are kept as well.
void mag_fwd(mhd_ctx* c, StepTape& t, const double* rho, double fac) {
  const size_t N = c->N;
  const int res = resistive(c);
  double* chol = t.chol ? t.chol : c->chol;
  if (res) {  // A.R. coefficient from the state entering the substep
    stab_eta(c->p, c->k, rho, t.Y[0], t.Y[0] + 4 * N, c->T, c->M, c->prm, t.eta, c->work, c->st);
    c->launches += kArLaunches;
  }
  if (c->prm.oe_vel) {
    stab_vel_prep(c->p, rho, chol, c->T, c->M, c->st);
    c->launches++;
  }
  for (int s = 0; s < 3; ++s) {
    double* in = t.Y[s];
    double* out = t.Y[s + 1];
    mag_stage(c->p, c->k, 1, in + 4 * N, in + N, in, rho, t.eta, res, t.Y[0] + 4 * N, t.Y[0] + N, t.Y[0],
              out + 4 * N, out + N, out, c->LJ, c->LE, c->T, c->M, c->dt, fac, RK_A[s], RK_B[s], s == 0, 0, c->st);
    c->launches += 3;
    if (c->prm.oe_vel) {
      cudaMemcpyAsync(t.vstar + 3 * N * s, out + N, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      stab_vel(c->p, c->k, rho, out, out + 4 * N, chol, c->T, c->M, c->prm, c->dt, fac, c->work,
               t.vfrz + (size_t)s * c->M.K * c->n, c->st);
      c->launches += kStatsLaunches + 1;
    }
  }
}

// One Strang step from the tape's input (U in hS[0][0], B in Y[0]), recording
// its stages; the end state goes to outU [5N] and, if non-null, outB [3Z].
void step_fwd(mhd_ctx* c, StepTape& t, double* outU, double* outB) {
  const size_t N = c->N;
  hydro_fwd(c, t, t.Ua, 0.5, 0);
  cons_to_prim(t.Ua, t.Y[0], N, c->st);
  mag_fwd(c, t, t.Ua, 1.0);
  cudaMemcpyAsync(t.hS[1][0], t.Ua, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  prim_to_cons(t.Y[3], t.hS[1][0], N, c->st);
  hydro_fwd(c, t, outU, 0.5, 1);
  if (outB) cudaMemcpyAsync(outB, t.Y[3] + 4 * N, 3 * c->Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  c->launches += 2;
}

// ---- adjoint substeps --------------------------------------------------------------
void hydro_adj(mhd_ctx* c, StepTape& t, double* lam, double tau, int h) {
  AdjBufs& A = c->adj;
  const size_t n = 5 * c->N;
  for (int s = 2; s >= 0; --s) {
    if (stab_on(c)) {  // stage map with frozen coefficients: lam <- P^T lam
      stab_hydro_adjoint(c->p, lam, frz_slot(c, t, h, s), c->T, c->M, c->prm.oe_hydro, c->prm.pp, c->st);
      c->launches++;
    }
    const double* w = lam;
    if (s > 0) {
      k_lin2<<<nblk(n), 256, 0, c->st>>>(lam, RK_A[s], RK_B[s], s == 1, A.L0, A.W, n);
      w = A.W;
    }
    hydro_rhs_vjp(c->p, t.hS[h][s], w, A.FA, A.G, c->M, c->T, c->st);
    k_fin<<<nblk(n), 256, 0, c->st>>>(w, A.G, tau, s == 0, s > 0 ? lam : A.L0, n);
    c->launches += s > 0 ? 4 : 3;
  }
  cudaMemcpyAsync(lam, A.L0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
}

void mag_adj(mhd_ctx* c, StepTape& t, const double* rho, double* lam, double tau) {
  AdjBufs& A = c->adj;
  const size_t N = c->N, n = 4 * N + 3 * c->Z;
  const double* chol = t.chol ? t.chol : c->chol;
  for (int s = 2; s >= 0; --s) {
    if (c->prm.oe_vel) {  // velocity OE with frozen coefficients: lam <- V^T lam
      stab_vel_adjoint(c->p, rho, lam, t.vstar + 3 * N * s, chol, t.vfrz + (size_t)s * c->M.K * c->n, c->T,
                       c->M, c->st);
      c->launches++;
    }
    const double* w = lam;
    if (s > 0) {
      k_lin2<<<nblk(n), 256, 0, c->st>>>(lam, RK_A[s], RK_B[s], s == 1, A.L0, A.W, n);
      w = A.W;
    }
    cudaMemsetAsync(A.G, 0, N * sizeof(double), c->st);  // no residual of e depends on e
    const double* Ys = t.Y[s];
    mag_rhs_vjp(c->p, c->k, rho, Ys + N, Ys + 4 * N, w, w + N, w + 4 * N, resistive(c) ? t.eta : nullptr, A.G + N,
                A.G + 4 * N, A.lamR, tau, A.ms, c->M, c->st);
    k_fin<<<nblk(n), 256, 0, c->st>>>(w, A.G, tau, s == 0, s > 0 ? lam : A.L0, n);
    c->launches += (s > 0 ? 2 : 1) + 9;
  }
  cudaMemcpyAsync(lam, A.L0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
}

// Backwards through one recorded step: lamU / the B part of lamM hold the
// adjoint of the step's end state and receive that of its start state.
void step_adj(mhd_ctx* c, StepTape& t, double dt) {
  AdjBufs& A = c->adj;
  const size_t N = c->N;
  hydro_adj(c, t, A.lamU, 0.5 * dt, 1);
  adj_prim_to_cons(t.hS[1][0], t.Y[3], A.lamU, A.lamM, A.lamR, N, c->st);
  mag_adj(c, t, t.Ua, A.lamM, dt);
  adj_cons_to_prim(t.Ua, A.lamM, A.lamR, A.lamU, N, c->st);
  hydro_adj(c, t, A.lamU, 0.5 * dt, 0);
  c->launches += 2;
}

// Packed host-layout vector (host or device) -> U [5N] and blocked B [3Z].
cudaError_t unpack_in(mhd_ctx* c, const double* x, double* U, double* B, int on_device) {
  AdjBufs& A = c->adj;
  const size_t N = c->N, Z = c->Z;
  cudaError_t e = acopy(c, A.io, x, 5 * N + 3 * Z, cudaMemcpyHostToDevice, on_device);
  if (e != cudaSuccess) return e;
  cudaMemcpyAsync(U, A.io, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  grid_to_blocked(A.io + 5 * N, B, c->M.nx, c->M.ny, c->mm, c->st);
  grid_to_blocked(A.io + 5 * N + Z, B + Z, c->M.nx, c->M.ny, c->mm, c->st);
  c->launches += 2;
  return cudaMemcpyAsync(B + 2 * Z, A.io + 5 * N + 2 * Z, Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
}

cudaError_t pack_out(mhd_ctx* c, const double* U, const double* B, double* x, int on_device) {
  AdjBufs& A = c->adj;
  const size_t N = c->N, Z = c->Z;
  cudaMemcpyAsync(A.io, U, 5 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  blocked_to_grid(B, A.io + 5 * N, c->M.nx, c->M.ny, c->mm, c->st);
  blocked_to_grid(B + Z, A.io + 5 * N + Z, c->M.nx, c->M.ny, c->mm, c->st);
  c->launches += 2;
  cudaMemcpyAsync(A.io + 5 * N + 2 * Z, B + 2 * Z, Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  return acopy(c, x, A.io, 5 * N + 3 * Z, cudaMemcpyDeviceToHost, on_device);
}

int read_status(mhd_ctx* c, unsigned* st) {
  cudaError_t e = cudaMemcpyAsync(c->h_status, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return acuda(e, "adjoint");
  *st = *c->h_status;
  return MHD_OK;
}

int stab_flags(const mhd_ctx* c) {
  return (c->prm.oe_hydro ? 1 : 0) | (c->prm.pp ? 2 : 0) | (c->prm.ar && c->prm.C_eta != 0.0 ? 4 : 0) |
         (c->prm.oe_vel ? 8 : 0);
}
const int kFrozenSupported = 1 | 2 | 4 | 8;  // every stabilisation map, with frozen coefficients

}  // namespace

extern "C" {

long long mhd_state_size(const mhd_ctx* c) { return c ? (long long)(5 * c->N + 3 * c->Z) : 0; }

// Common checks and set-up of the adjoint calls.
static int adjoint_begin(mhd_ctx* c, double dt, int* flags) {
  const int fl = stab_flags(c);
  if (flags) *flags = fl;
  if (c->prm.strang_order != 0) return afail(MHD_EINVAL, "the adjoint differentiates the H-M-H step");
  if (fl & ~kFrozenSupported) return afail(MHD_EINVAL, "unsupported stabilisation map");
  if (!(dt > 0.0)) return afail(MHD_EINVAL, "dt must be positive");
  return ensure_adjoint(c);
}

static int recompute_status(mhd_ctx* c) {
  unsigned st = 0;
  int r = read_status(c, &st);
  if (r != MHD_OK) return r;
  if (st & ST_NONFINITE) return afail(MHD_NONFINITE, "non-finite value in the recomputed steps");
  if (st & ST_INADMISSIBLE) return afail(MHD_INADMISSIBLE, "inadmissible cell average in the recomputed steps");
  return MHD_OK;
}

int mhd_adjoint_step(mhd_ctx* c, const double* state_n, const double* lam_np1, double* lam_n, double dt,
                     int on_device, int* flags) {
  return mhd_adjoint_segment(c, state_n, 1, lam_np1, lam_n, dt, on_device, flags);
}

int mhd_adjoint_segment(mhd_ctx* c, const double* state_0, int nsteps, const double* lam_end, double* lam_0,
                        double dt, int on_device, int* flags) {
  if (!c || !state_0 || !lam_end || !lam_0 || nsteps < 1) return afail(MHD_EINVAL, "invalid argument");
  int r = adjoint_begin(c, dt, flags);
  if (r != MHD_OK) return r;
  if ((r = ensure_tapes(c, nsteps)) != MHD_OK) return r;
  AdjBufs& A = c->adj;
  const size_t N = c->N;
  cudaError_t e;
  // forward: record every step of the segment
  if ((e = unpack_in(c, state_0, A.tapes[0].hS[0][0], A.tapes[0].Y[0] + 4 * N, on_device)) != cudaSuccess)
    return acuda(e, "adjoint state");
  set_scalar(c->dt, dt, c->st);
  cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->st);
  for (int i = 0; i < nsteps; ++i) {
    const bool last = i + 1 == nsteps;
    step_fwd(c, A.tapes[i], last ? A.G : A.tapes[i + 1].hS[0][0], last ? nullptr : A.tapes[i + 1].Y[0] + 4 * N);
  }
  if ((r = recompute_status(c)) != MHD_OK) return r;
  // backward
  if ((e = unpack_in(c, lam_end, A.lamU, A.lamM + 4 * N, on_device)) != cudaSuccess)
    return acuda(e, "adjoint input");
  for (int i = nsteps - 1; i >= 0; --i) step_adj(c, A.tapes[i], dt);
  if ((e = pack_out(c, A.lamU, A.lamM + 4 * N, lam_0, on_device)) != cudaSuccess) return acuda(e, "adjoint output");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return acuda(e, "adjoint");
  return MHD_OK;
}

int mhd_hydro_rhs_vjp(mhd_ctx* c, const double* U, const double* nu, double* out, int on_device) {
  if (!c || !U || !nu || !out) return afail(MHD_EINVAL, "null argument");
  int r = ensure_adjoint(c);
  if (r != MHD_OK) return r;
  AdjBufs& A = c->adj;
  StepTape& t = A.tapes[0];
  const size_t n = 5 * c->N;
  cudaError_t e;
  if ((e = acopy(c, t.hS[0][0], U, n, cudaMemcpyHostToDevice, on_device)) != cudaSuccess) return acuda(e, "U");
  if ((e = acopy(c, A.W, nu, n, cudaMemcpyHostToDevice, on_device)) != cudaSuccess) return acuda(e, "nu");
  hydro_rhs_vjp(c->p, t.hS[0][0], A.W, A.FA, A.G, c->M, c->T, c->st);
  c->launches += 2;
  if ((e = acopy(c, out, A.G, n, cudaMemcpyDeviceToHost, on_device)) != cudaSuccess) return acuda(e, "out");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return acuda(e, "hydro_rhs_vjp");
  return MHD_OK;
}

int mhd_mag_rhs_vjp(mhd_ctx* c, const double* rho, const double* u, const double* Bx, const double* By,
                    const double* Bz, const double* wu, const double* wBx, const double* wBy, const double* wBz,
                    double* g_rho, double* g_u, double* g_Bx, double* g_By, double* g_Bz, int on_device) {
  if (!c || !rho || !u || !Bx || !By || !Bz || !wu || !wBx || !wBy || !wBz || !g_rho || !g_u || !g_Bx || !g_By ||
      !g_Bz)
    return afail(MHD_EINVAL, "null argument");
  int r = ensure_adjoint(c);
  if (r != MHD_OK) return r;
  AdjBufs& A = c->adj;
  const size_t N = c->N, Z = c->Z;
  const int nx = c->M.nx, ny = c->M.ny, mm = c->mm;
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
  StepTape& t = A.tapes[0];
  double* Y = t.Y[0];
  double* io = A.io;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = acopy(c, t.Ua, rho, N, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, Y + N, u, 3 * N, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, io, Bx, Z, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, io + Z, By, Z, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, Y + 4 * N + 2 * Z, Bz, Z, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, A.W + N, wu, 3 * N, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, io + 2 * Z, wBx, Z, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, io + 3 * Z, wBy, Z, h2d, on_device);
  if (e == cudaSuccess) e = acopy(c, A.W + 4 * N + 2 * Z, wBz, Z, h2d, on_device);
  if (e != cudaSuccess) return acuda(e, "mag_rhs_vjp inputs");
  grid_to_blocked(io, Y + 4 * N, nx, ny, mm, c->st);
  grid_to_blocked(io + Z, Y + 4 * N + Z, nx, ny, mm, c->st);
  grid_to_blocked(io + 2 * Z, A.W + 4 * N, nx, ny, mm, c->st);
  grid_to_blocked(io + 3 * Z, A.W + 4 * N + Z, nx, ny, mm, c->st);
  cudaMemsetAsync(A.lamR, 0, N * sizeof(double), c->st);
  mag_rhs_vjp(c->p, c->k, t.Ua, Y + N, Y + 4 * N, nullptr, A.W + N, A.W + 4 * N, nullptr, A.G + N, A.G + 4 * N,
              A.lamR, 1.0, A.ms, c->M, c->st);
  blocked_to_grid(A.G + 4 * N, io, nx, ny, mm, c->st);
  blocked_to_grid(A.G + 4 * N + Z, io + Z, nx, ny, mm, c->st);
  c->launches += 15;
  if (e == cudaSuccess) e = acopy(c, g_rho, A.lamR, N, d2h, on_device);
  if (e == cudaSuccess) e = acopy(c, g_u, A.G + N, 3 * N, d2h, on_device);
  if (e == cudaSuccess) e = acopy(c, g_Bx, io, Z, d2h, on_device);
  if (e == cudaSuccess) e = acopy(c, g_By, io + Z, Z, d2h, on_device);
  if (e == cudaSuccess) e = acopy(c, g_Bz, A.G + 4 * N + 2 * Z, Z, d2h, on_device);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return acuda(e, "mag_rhs_vjp");
  return MHD_OK;
}

}  // extern "C"
