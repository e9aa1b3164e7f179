// C ABI of the library (include/mhd.h): context, state transfer and the
// Strang driver (Algorithm 3) with the raw-average rejection and retry of the
// hydro stage (§3.2.3).  All work is enqueued on one stream; the host reads
// one status word per step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "context.cuh"


using namespace mhd;

namespace {
thread_local std::string g_err;
}  // namespace

// Lets the allocation-free entry point report through mhd_last_error().
void mhd::set_error_message(const char* msg) { g_err = msg; }

namespace {

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
const char* const kNotPlanar = "reduced_2d2v needs u_z = B_z = 0 (a nonzero m_z or B_z was found; state restored)";
int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return MHD_ECUDA;
}
}  // namespace


namespace {

cudaError_t dalloc(mhd_ctx* c, double** p, size_t n) {
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(n, 1) * sizeof(double));
  if (e == cudaSuccess) { c->allocs.push_back(ptr); *p = (double*)ptr; }
  return e;
}

cudaError_t copy_in(mhd_ctx* c, double* dst, const double* src, size_t n, int on_device) {
  if (on_device) return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->st);
}
cudaError_t copy_out(mhd_ctx* c, double* dst, const double* src, size_t n, int on_device) {
  if (on_device) return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->st);
}

// Kernel classes of the event profiler.
enum { KC_FACE = 0, KC_VOL, KC_MAG_J, KC_MAG_E, KC_MAG_B, KC_EXCH, KC_STAB_H, KC_STAB_ETA, KC_STAB_VEL, KC_COUNT };

// Scoped event pair around the launches of one kernel class.
struct Prof {
  mhd_ctx* c;
  int kc;
  cudaEvent_t a, b;
  Prof(mhd_ctx* c_, int kc_) : c(c_), kc(kc_), a(nullptr), b(nullptr) {
    if (!c->profiling) return;
    size_t used = 2 * c->ev_rec.size();
    while (c->ev_pool.size() < used + 2) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->ev_pool.push_back(e);
    }
    a = c->ev_pool[used];
    b = c->ev_pool[used + 1];
    c->ev_rec.push_back({kc, {a, b}});
    cudaEventRecord(a, c->st);
  }
  ~Prof() {
    if (a) cudaEventRecord(b, c->st);
  }
};

const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};
const double RK_B[3] = {1.0, 0.25, 2.0 / 3.0};

// Hydro substep Phi_H^{tau}, tau = dt * fac (Algorithm 1).
void hydro_substep(mhd_ctx* c, double fac) {
  const double* in[3] = {c->U, c->S1, c->S2};
  double* out[3] = {c->S1, c->S2, c->U};
  bool stab = c->prm.oe_hydro || c->prm.pp;
  // With the limiter on, its own test of the element averages of the OE output
  // (which keeps the raw averages) is the admissibility check (§3.2.3, reading
  // R9): the volume kernel then skips its raw-average reduction.
  unsigned* vol_status = c->prm.pp ? nullptr : c->status;
  for (int s = 0; s < 3; ++s) {
    { Prof pr(c, KC_FACE); hydro_face(c->p, in[s], c->Fx, c->Fy, c->M, c->st); }
    { Prof pr(c, KC_VOL);
      hydro_vol(c->p, 1, in[s], c->U, c->Fx, c->Fy, out[s], nullptr, vol_status, c->T, c->M, c->dt, fac, RK_A[s],
                RK_B[s], s == 0, c->st); }
    c->launches += 2;
    if (stab) {
      Prof pr(c, KC_STAB_H);
      stab_hydro(c->p, out[s], c->status, c->T, c->M, c->prm, c->dt, fac, c->work, nullptr, c->st);
      c->launches += c->prm.oe_hydro ? kStatsLaunches + 1 : 1;
    }
  }
}

// Magnetic substep Phi_M^{tau}, tau = dt * fac (Algorithm 2), with the nodal
// exchange before and after (§3.4.1).
void mag_substep(mhd_ctx* c, double fac) {
  const size_t N = c->N;
  if (c->prm.reduced) {  // the reduced stage is exact only for u_z = B_z = 0
    check_planar(c->U + 3 * N, N, c->B + 2 * c->Z, c->Z, c->status, c->st);
    c->launches++;
  }
  { Prof pr(c, KC_EXCH); cons_to_prim(c->U, c->Y0, N, c->st); }
  c->launches++;
  int resistive = c->prm.ar && c->prm.C_eta != 0.0;
  if (resistive) {
    Prof pr(c, KC_STAB_ETA);
    stab_eta(c->p, c->k, c->U, c->Y0, c->B, c->T, c->M, c->prm, c->eta, c->work, c->st);
    c->launches += kArLaunches;
  } else {
    cudaMemsetAsync(c->eta, 0, c->M.K * sizeof(double), c->st);
  }
  if (c->prm.oe_vel) {
    Prof pr(c, KC_STAB_VEL);
    stab_vel_prep(c->p, c->U, c->chol, c->T, c->M, c->st);
    c->launches++;
  }
  const double* Bin[3] = {c->B, c->Ba, c->Bb};
  double* Bout[3] = {c->Ba, c->Bb, c->B};
  const double* Yin[3] = {c->Y0, c->Ya, c->Yb};
  double* Yout[3] = {c->Ya, c->Yb, c->Y0};
  for (int s = 0; s < 3; ++s) {
    {
      Prof pr(c, KC_MAG_E);
      mag_stage(c->p, c->k, 1, Bin[s], Yin[s] + N, Yin[s], c->U, c->eta, resistive, c->B, c->Y0 + N, c->Y0,
                Bout[s], Yout[s] + N, Yout[s], c->LJ, c->LE, c->T, c->M, c->dt, fac, RK_A[s], RK_B[s], s == 0,
                c->prm.reduced, c->st);
    }
    c->launches += 3;
    if (c->prm.oe_vel) {
      Prof pr(c, KC_STAB_VEL);
      stab_vel(c->p, c->k, c->U, Yout[s], Bout[s], c->chol, c->T, c->M, c->prm, c->dt, fac, c->work, nullptr,
               c->st);
      c->launches += kStatsLaunches + 1;
    }
  }
  Prof pr(c, KC_EXCH);
  prim_to_cons(c->Y0, c->U, N, c->st);
  c->launches++;
}

// One Strang step (Algorithm 3, eq. strang-composition): H-M-H, or the
// M-H-M ordering when requested.
void enqueue_strang(mhd_ctx* c) {
  if (c->prm.strang_order == 1) {
    mag_substep(c, 0.5);
    hydro_substep(c, 1.0);
    mag_substep(c, 0.5);
    return;
  }
  hydro_substep(c, 0.5);
  mag_substep(c, 1.0);
  hydro_substep(c, 0.5);
}

int check_status(mhd_ctx* c, unsigned* st_out) {
  cudaError_t e = cudaMemcpyAsync(c->h_status, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(e, "step");
  *st_out = *c->h_status;
  return MHD_OK;
}

}  // namespace

namespace mhd {
unsigned long long oob_hydro(bool reset);
unsigned long long oob_stab(bool reset);
unsigned long long oob_magnetic(bool reset);
unsigned long long oob_misc(bool reset);
}  // namespace mhd

extern "C" {

const char* mhd_last_error(void) { return g_err.c_str(); }

long long mhd_debug_oob(int reset) {
#ifdef MHD_BOUNDS_CHECK
  cudaDeviceSynchronize();
  return (long long)(oob_hydro(reset) + oob_stab(reset) + oob_magnetic(reset) + oob_misc(reset));
#else
  (void)reset;
  return -1;
#endif
}

const char* mhd_status_string(int s) {
  switch (s) {
    case MHD_OK: return "ok";
    case MHD_RETRIED: return "step retried with a smaller dt";
    case MHD_EINVAL: return "invalid argument";
    case MHD_ENOMEM: return "out of device memory";
    case MHD_ECUDA: return "CUDA error";
    case MHD_INADMISSIBLE: return "inadmissible cell average after all halvings";
    case MHD_NONFINITE: return "non-finite value";
    case MHD_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

int mhd_create(const mhd_mesh_t* mesh, int p, int k, double gamma, mhd_ctx** out) {
  if (!mesh || !out) return fail(MHD_EINVAL, "null argument");
  *out = nullptr;
  if (mesh->nx < 1 || mesh->ny < 1 || !(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0))
    return fail(MHD_EINVAL, "invalid mesh");
  if (table_slot(p, k) < 0) return fail(MHD_EINVAL, "unsupported (p, k): need 1 <= p <= 4 and k in {p-1, p}");
  if (!(gamma > 1.0)) return fail(MHD_EINVAL, "gamma must exceed 1");
  if ((long long)mesh->nx * mesh->ny > (1LL << 30)) return fail(MHD_EINVAL, "mesh too large");
  mhd_ctx* c = new (std::nothrow) mhd_ctx();
  if (!c) return fail(MHD_ENOMEM, "host allocation");
  c->p = p; c->k = k; c->n = p + 1; c->n2 = c->n * c->n; c->mm = k + 1;
  c->x0 = mesh->x0; c->x1 = mesh->x1; c->y0 = mesh->y0; c->y1 = mesh->y1;
  c->M.nx = mesh->nx; c->M.ny = mesh->ny; c->M.K = mesh->nx * mesh->ny;
  c->M.hx = (mesh->x1 - mesh->x0) / mesh->nx;
  c->M.hy = (mesh->y1 - mesh->y0) / mesh->ny;
  c->M.Jdet = c->M.hx * c->M.hy / 4.0;
  c->M.g = gamma;
  mesh_reciprocals(c->M);
  c->prm = Stab{0, 0, 0, 0, 0.02, 0.02, 5.0, 0.2, 0.4, 20};
  c->N = (size_t)c->M.K * c->n2;
  c->Z = (size_t)c->M.K * c->mm * c->mm;
  c->launches = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "stream"); }
  c->own_stream = true;
  c->T = device_tables(p, k, &e);
  if (!c->T) { cudaStreamDestroy(c->st); delete c; return cuda_fail(e, "tables"); }
  if ((e = mag_prepare(p, k)) != cudaSuccess || (e = stab_prepare(p)) != cudaSuccess ||
      (e = mag_adj_prepare(p, k)) != cudaSuccess) {
    cudaStreamDestroy(c->st);
    delete c;
    return cuda_fail(e, "kernel attributes");
  }
  host_tables(p, k, &c->hT);
  const size_t N = c->N, Z = c->Z, K = c->M.K;
  double** bufs5[] = {&c->U, &c->Usave, &c->S1, &c->S2};
  for (auto b : bufs5) if ((e = dalloc(c, b, 5 * N)) != cudaSuccess) goto oom;
  {
    double** bufs3[] = {&c->B, &c->Bsave, &c->Ba, &c->Bb};
    for (auto b : bufs3) if ((e = dalloc(c, b, 3 * Z)) != cudaSuccess) goto oom;
    double** bufs4[] = {&c->Y0, &c->Ya, &c->Yb};
    for (auto b : bufs4) if ((e = dalloc(c, b, 4 * N)) != cudaSuccess) goto oom;
  }
  if ((e = dalloc(c, &c->Fx, 5 * K * c->n)) != cudaSuccess) goto oom;
  if ((e = dalloc(c, &c->Fy, 5 * K * c->n)) != cudaSuccess) goto oom;
  if ((e = dalloc(c, &c->LJ, mag_load_doubles(p, k, (int)K))) != cudaSuccess) goto oom;
  if ((e = dalloc(c, &c->LE, mag_load_doubles(p, k, (int)K))) != cudaSuccess) goto oom;
  if ((e = dalloc(c, &c->eta, K)) != cudaSuccess) goto oom;
  if ((e = dalloc(c, &c->dt, 4)) != cudaSuccess) goto oom;
  if ((e = dalloc(c, &c->work, std::max(stab_work_doubles(p, k, c->M), 12 * K))) != cudaSuccess) goto oom;
  if ((e = dalloc(c, &c->chol, stab_chol_doubles(p, c->M))) != cudaSuccess) goto oom;
  if ((e = stab_init_mesh(p, c->hT, c->M, c->work)) != cudaSuccess) { mhd_destroy(c); return cuda_fail(e, "mesh coefficients"); }
  if ((e = dalloc(c, &c->io, std::max(5 * N, 3 * Z + 4 * N))) != cudaSuccess) goto oom;
  {
    void* ptr = nullptr;
    if ((e = cudaMalloc(&ptr, 64)) != cudaSuccess) goto oom;
    c->allocs.push_back(ptr);
    c->status = (unsigned*)ptr;
    c->prm.activity = c->status + 1;
    c->maxbits = (unsigned long long*)((char*)ptr + 16);
    if ((e = cudaMallocHost(&ptr, 64)) != cudaSuccess) goto oom;
    c->h_pinned = (double*)ptr;
    c->h_status = (unsigned*)((char*)ptr + 32);
  }
  cudaMemsetAsync(c->U, 0, 5 * N * sizeof(double), c->st);
  cudaMemsetAsync(c->B, 0, 3 * Z * sizeof(double), c->st);
  cudaMemsetAsync(c->eta, 0, K * sizeof(double), c->st);
  cudaMemsetAsync(c->status, 0, 64, c->st);
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) { mhd_destroy(c); return cuda_fail(e, "init"); }
  *out = c;
  return MHD_OK;
oom:
  mhd_destroy(c);
  return fail(MHD_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
}

int mhd_create_walled(const mhd_mesh_t* mesh, int p, int k, double gamma, int walls, int conducting,
                      mhd_ctx** out) {
  if (!mesh || !out) return fail(MHD_EINVAL, "null argument");
  *out = nullptr;
  if (walls < 1 || walls > 3 || conducting < 0 || conducting > 3 || (conducting & ~walls))
    return fail(MHD_EINVAL, "walls must be 1 (x), 2 (y) or 3; conducting a subset of the walled directions");
  if (mesh->nx < 1 || mesh->ny < 1 || !(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0))
    return fail(MHD_EINVAL, "invalid mesh");
  if ((long long)mesh->nx * mesh->ny * ((walls & 1) ? 2 : 1) * ((walls & 2) ? 2 : 1) > (1LL << 30))
    return fail(MHD_EINVAL, "mesh too large");
  mhd_mesh_t m2 = *mesh;
  if (walls & 1) { m2.nx = 2 * mesh->nx; m2.x1 = 2.0 * mesh->x1 - mesh->x0; }
  if (walls & 2) { m2.ny = 2 * mesh->ny; m2.y1 = 2.0 * mesh->y1 - mesh->y0; }
  int r = mhd_create(&m2, p, k, gamma, out);
  if (r != MHD_OK) return r;
  (*out)->walls = walls;
  (*out)->cond = conducting;
  (*out)->pnx = mesh->nx;
  (*out)->pny = mesh->ny;
  return MHD_OK;
}

int mhd_mirror_fill(mhd_ctx* c) {
  if (!c) return fail(MHD_EINVAL, "null context");
  if (!c->walls) return fail(MHD_EINVAL, "not a walled context (mhd_create_walled)");
  mirror_fill(c->p, c->k, c->U, c->B, c->M, c->pnx, c->pny, c->walls, c->cond, c->st);
  c->launches += 2;
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(e, "mirror_fill");
  return MHD_OK;
}

void mhd_destroy(mhd_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

int mhd_set_params(mhd_ctx* c, const mhd_params_t* prm) {
  if (!c || !prm) return fail(MHD_EINVAL, "null argument");
  if (prm->s_H < 0 || prm->s_M < 0 || prm->C_s < 0 || prm->C_eta < 0 || !(prm->cfl > 0) || prm->max_halvings < 0 ||
      (prm->strang_order != 0 && prm->strang_order != 1) || (prm->reduced_2d2v != 0 && prm->reduced_2d2v != 1))
    return fail(MHD_EINVAL, "invalid stabilisation parameters");
  c->prm = Stab{prm->oe_hydro, prm->oe_vel, prm->pp, prm->ar, prm->s_H, prm->s_M, prm->C_s, prm->C_eta, prm->cfl,
                prm->max_halvings, c->status + 1, prm->strang_order, prm->reduced_2d2v};
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return MHD_OK;
}

int mhd_set_stream(mhd_ctx* c, void* stream) {
  if (!c) return fail(MHD_EINVAL, "null context");
  cudaStreamSynchronize(c->st);
  if (c->own_stream) cudaStreamDestroy(c->st);
  c->st = (cudaStream_t)stream;
  c->own_stream = false;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return MHD_OK;
}

int mhd_sizes(const mhd_ctx* c, long long* K, long long* N, long long* G, long long* Z) {
  if (!c) return fail(MHD_EINVAL, "null context");
  if (K) *K = c->M.K;
  if (N) *N = (long long)c->N;
  if (G) *G = (long long)c->Z;
  if (Z) *Z = (long long)c->Z;
  return MHD_OK;
}

int mhd_node_coords(const mhd_ctx* c, int which, double* X, double* Y) {
  if (!c || !X || !Y) return fail(MHD_EINVAL, "null argument");
  const Tab& T = c->hT;
  const int nx = c->M.nx, ny = c->M.ny, n = c->n, mm = c->mm;
  for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
      double xl = c->x0 + ex * c->M.hx, yl = c->y0 + ey * c->M.hy;
      size_t k = (size_t)ey * nx + ex;
      if (which == 0) {
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            X[k * n * n + j * n + i] = xl + 0.5 * (1.0 + T.xp[i]) * c->M.hx;
            Y[k * n * n + j * n + i] = yl + 0.5 * (1.0 + T.xp[j]) * c->M.hy;
          }
      } else if (which == 1) {
        for (int b = 0; b < mm; ++b)
          for (int a = 0; a < mm; ++a) {
            size_t g = (size_t)(ey * mm + b) * nx * mm + ex * mm + a;
            X[g] = xl + 0.5 * (1.0 + T.xL[a]) * c->M.hx;
            Y[g] = yl + 0.5 * (1.0 + T.xL[b]) * c->M.hy;
          }
      } else if (which == 2) {
        for (int b = 0; b < mm; ++b)
          for (int a = 0; a < mm; ++a) {
            X[k * mm * mm + b * mm + a] = xl + 0.5 * (1.0 + T.xM[a]) * c->M.hx;
            Y[k * mm * mm + b * mm + a] = yl + 0.5 * (1.0 + T.xM[b]) * c->M.hy;
          }
      } else {
        return fail(MHD_EINVAL, "which must be 0, 1 or 2");
      }
    }
  return MHD_OK;
}

int mhd_set_state(mhd_ctx* c, const double* U, const double* Bx, const double* By, const double* Bz, int on_device) {
  if (!c || !U || !Bx || !By || !Bz) return fail(MHD_EINVAL, "null argument");
  cudaError_t e;
  if ((e = copy_in(c, c->U, U, 5 * c->N, on_device)) != cudaSuccess) return cuda_fail(e, "set_state U");
  if ((e = copy_in(c, c->io, Bx, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "set_state Bx");
  grid_to_blocked(c->io, c->B, c->M.nx, c->M.ny, c->mm, c->st);
  if ((e = copy_in(c, c->io, By, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "set_state By");
  grid_to_blocked(c->io, c->B + c->Z, c->M.nx, c->M.ny, c->mm, c->st);
  if ((e = copy_in(c, c->B + 2 * c->Z, Bz, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "set_state Bz");
  c->launches += 2;
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "set_state");
  return MHD_OK;
}

int mhd_get_state(mhd_ctx* c, double* U, double* Bx, double* By, double* Bz, int on_device) {
  if (!c) return fail(MHD_EINVAL, "null context");
  cudaError_t e;
  if (U && (e = copy_out(c, U, c->U, 5 * c->N, on_device)) != cudaSuccess) return cuda_fail(e, "get_state U");
  if (Bx) {
    blocked_to_grid(c->B, c->io, c->M.nx, c->M.ny, c->mm, c->st);
    c->launches++;
    if ((e = copy_out(c, Bx, c->io, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "get_state Bx");
    if (on_device && (e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "get_state");
  }
  if (By) {
    blocked_to_grid(c->B + c->Z, c->io, c->M.nx, c->M.ny, c->mm, c->st);
    c->launches++;
    if ((e = copy_out(c, By, c->io, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "get_state By");
    if (on_device && (e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "get_state");
  }
  if (Bz && (e = copy_out(c, Bz, c->B + 2 * c->Z, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "get_state Bz");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "get_state");
  return MHD_OK;
}

int mhd_set_primitive(mhd_ctx* c, const double* rho, const double* u, const double* p, int on_device) {
  if (!c || !rho || !u || !p) return fail(MHD_EINVAL, "null argument");
  const size_t N = c->N;
  cudaError_t e;
  if ((e = copy_in(c, c->io, rho, N, on_device)) != cudaSuccess) return cuda_fail(e, "rho");
  if ((e = copy_in(c, c->io + N, u, 3 * N, on_device)) != cudaSuccess) return cuda_fail(e, "u");
  if ((e = copy_in(c, c->S1, p, N, on_device)) != cudaSuccess) return cuda_fail(e, "p");
  prim_in(c->io, c->io + N, c->S1, c->U, N, c->M.g, c->st);
  c->launches++;
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "set_primitive");
  return MHD_OK;
}

int mhd_primitive_to_conservative(mhd_ctx* c, const double* rho, const double* u, const double* p, double* U,
                                  int on_device) {
  if (!c || !rho || !u || !p || !U) return fail(MHD_EINVAL, "null argument");
  const size_t N = c->N;
  cudaError_t e;
  if ((e = copy_in(c, c->io, rho, N, on_device)) != cudaSuccess) return cuda_fail(e, "rho");
  if ((e = copy_in(c, c->io + N, u, 3 * N, on_device)) != cudaSuccess) return cuda_fail(e, "u");
  if ((e = copy_in(c, c->io + 4 * N, p, N, on_device)) != cudaSuccess) return cuda_fail(e, "p");
  prim_in(c->io, c->io + N, c->io + 4 * N, c->S1, N, c->M.g, c->st);
  c->launches++;
  if ((e = copy_out(c, U, c->S1, 5 * N, on_device)) != cudaSuccess) return cuda_fail(e, "U");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "primitive_to_conservative");
  return MHD_OK;
}

int mhd_primitive_to_conservative_vjp(mhd_ctx* c, const double* rho, const double* u, const double* lamU,
                                      double* g_rho, double* g_u, double* g_p, int on_device) {
  if (!c || !rho || !u || !lamU || !g_rho || !g_u || !g_p) return fail(MHD_EINVAL, "null argument");
  const size_t N = c->N;
  cudaError_t e;
  if ((e = copy_in(c, c->io, rho, N, on_device)) != cudaSuccess) return cuda_fail(e, "rho");
  if ((e = copy_in(c, c->io + N, u, 3 * N, on_device)) != cudaSuccess) return cuda_fail(e, "u");
  if ((e = copy_in(c, c->S1, lamU, 5 * N, on_device)) != cudaSuccess) return cuda_fail(e, "lamU");
  prim_in_vjp(c->io, c->io + N, c->S1, c->S2, N, c->M.ig1, c->st);
  c->launches++;
  if ((e = copy_out(c, g_rho, c->S2, N, on_device)) != cudaSuccess) return cuda_fail(e, "g_rho");
  if ((e = copy_out(c, g_u, c->S2 + N, 3 * N, on_device)) != cudaSuccess) return cuda_fail(e, "g_u");
  if ((e = copy_out(c, g_p, c->S2 + 4 * N, N, on_device)) != cudaSuccess) return cuda_fail(e, "g_p");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "primitive_to_conservative_vjp");
  return MHD_OK;
}

int mhd_set_B_from_potential(mhd_ctx* c, const double* Az, double Bx0, double By0, const double* Bz, int on_device) {
  if (!c || !Az || !Bz) return fail(MHD_EINVAL, "null argument");
  cudaError_t e;
  if ((e = copy_in(c, c->io, Az, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "Az");
  grid_to_blocked(c->io, c->io + c->Z, c->M.nx, c->M.ny, c->mm, c->st);
  b_from_potential(c->k, c->io + c->Z, Bx0, By0, c->B, c->B + c->Z, c->T, c->M, c->st);
  c->launches += 2;
  if ((e = copy_in(c, c->B + 2 * c->Z, Bz, c->Z, on_device)) != cudaSuccess) return cuda_fail(e, "Bz");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "set_B_from_potential");
  return MHD_OK;
}

int mhd_quad_coords(const mhd_ctx* c, int nq, double* X, double* Y) {
  if (!c || !X || !Y) return fail(MHD_EINVAL, "null argument");
  if (nq < 1 || nq > MHD_QMAX) return fail(MHD_EINVAL, "nq must be in [1, 16]");
  double z[MHD_QMAX];
  gauss_points(nq, z);
  const int nx = c->M.nx, ny = c->M.ny;
  for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
      double xl = c->x0 + ex * c->M.hx, yl = c->y0 + ey * c->M.hy;
      size_t base = ((size_t)ey * nx + ex) * nq * nq;
      for (int qy = 0; qy < nq; ++qy)
        for (int qx = 0; qx < nq; ++qx) {
          X[base + qy * nq + qx] = xl + 0.5 * (1.0 + z[qx]) * c->M.hx;
          Y[base + qy * nq + qx] = yl + 0.5 * (1.0 + z[qy]) * c->M.hy;
        }
    }
  return MHD_OK;
}

int mhd_set_Bz_projected(mhd_ctx* c, const double* fq, int nq, int on_device) {
  if (!c || !fq) return fail(MHD_EINVAL, "null argument");
  if (nq < c->k + 1 || nq > MHD_QMAX) return fail(MHD_EINVAL, "nq must be in [k+1, 16]");
  const size_t n = (size_t)c->M.K * nq * nq;
  cudaError_t e;
  double* tmp = nullptr;
  const double* src = fq;
  if (!on_device) {
    if ((e = cudaMalloc(&tmp, n * sizeof(double))) != cudaSuccess) return cuda_fail(e, "B_z data");
    if ((e = copy_in(c, tmp, fq, n, 0)) != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(e, "B_z data");
    }
    src = tmp;
  }
  l2_project(c->k, nq, src, c->B + 2 * c->Z, (size_t)c->M.K, c->st);
  c->launches++;
  e = cudaStreamSynchronize(c->st);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "set_Bz_projected");
  return MHD_OK;
}

int mhd_compute_dt(mhd_ctx* c, double* dt) {
  if (!c || !dt) return fail(MHD_EINVAL, "null argument");
  cfl_dt(c->p, c->k, c->U, c->B, c->T, c->M, c->maxbits, c->prm.cfl, c->dt, c->st);
  c->launches += 2;
  cudaError_t e = cudaMemcpyAsync(c->h_pinned, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(e, "compute_dt");
  *dt = c->h_pinned[0];
  if (!std::isfinite(*dt) || !(*dt > 0)) return fail(MHD_NONFINITE, "non-finite CFL step");
  return MHD_OK;
}

int mhd_strang_step(mhd_ctx* c, double dt, double* dt_taken) {
  if (!c) return fail(MHD_EINVAL, "null context");
  cudaError_t e;
  if (!(dt > 0)) {
    int r = mhd_compute_dt(c, &dt);
    if (r != MHD_OK) return r;
  }
  cudaMemcpyAsync(c->Usave, c->U, 5 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->Bsave, c->B, 3 * c->Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  for (int att = 0; att <= c->prm.max_halvings; ++att) {
    cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->st);
    set_scalar(c->dt, dt, c->st);
    c->launches++;
    enqueue_strang(c);
    unsigned s = 0;
    int r = check_status(c, &s);
    if (r != MHD_OK) return r;
    if (s & ST_NOT_PLANAR) {
      cudaMemcpyAsync(c->U, c->Usave, 5 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      cudaMemcpyAsync(c->B, c->Bsave, 3 * c->Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      cudaStreamSynchronize(c->st);
      return fail(MHD_EINVAL, kNotPlanar);
    }
    if (!(s & ST_INADMISSIBLE)) {
      if (dt_taken) *dt_taken = dt;
      return att > 0 ? MHD_RETRIED : MHD_OK;
    }
    cudaMemcpyAsync(c->U, c->Usave, 5 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(c->B, c->Bsave, 3 * c->Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    c->rejections++;
    dt *= 0.5;
  }
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "restore");
  if (dt_taken) *dt_taken = 0.0;
  return fail(MHD_INADMISSIBLE, "inadmissible cell average after all halvings");
}

// Capture `nsteps` Strang steps (state save included) on stream `st` of the
// context; the step length is read from the device word c->dt at run time.
static void enqueue_sequence(mhd_ctx* c, int nsteps) {
  cudaMemcpyAsync(c->Usave, c->U, 5 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->Bsave, c->B, 3 * c->Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
  for (int s = 0; s < nsteps; ++s) enqueue_strang(c);
}

// Instantiated graph of a fixed-dt sequence of nsteps Strang steps (cached).
static int sequence_graph(mhd_ctx* c, int nsteps) {
  if (c->graph && c->graph_steps == nsteps) return MHD_OK;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  cudaGraph_t g = nullptr;
  long long l0 = c->launches;
  cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "begin capture");
  enqueue_sequence(c, nsteps);
  e = cudaStreamEndCapture(c->st, &g);
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { c->graph = nullptr; return cuda_fail(e, "graph instantiate"); }
  c->graph_steps = nsteps;
  c->graph_launches = c->launches - l0;
  c->launches = l0;
  return MHD_OK;
}

static bool capturable(cudaStream_t s) {
  return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

int mhd_strang_steps(mhd_ctx* c, double dt, int nsteps, int* steps_done) {
  if (!c || !(dt > 0) || nsteps < 0) return fail(MHD_EINVAL, "invalid argument");
  if (steps_done) *steps_done = 0;
  if (nsteps == 0) return MHD_OK;
  // the legacy default stream cannot be captured, and the event profiler needs
  // the eager launches: run eagerly in both cases
  const bool graph = capturable(c->st) && !c->profiling;
  if (graph) {
    int r = sequence_graph(c, nsteps);
    if (r != MHD_OK) return r;
  }
  cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->st);
  set_scalar(c->dt, dt, c->st);
  c->launches++;
  if (graph) {
    cudaError_t e = cudaGraphLaunch(c->graph, c->st);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    c->launches += c->graph_launches;
  } else {
    enqueue_sequence(c, nsteps);
  }
  int r;
  unsigned s = 0;
  r = check_status(c, &s);
  if (r != MHD_OK) return r;
  if (s & (ST_INADMISSIBLE | ST_NOT_PLANAR)) {
    cudaMemcpyAsync(c->U, c->Usave, 5 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(c->B, c->Bsave, 3 * c->Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    cudaStreamSynchronize(c->st);
    if (s & ST_NOT_PLANAR) return fail(MHD_EINVAL, kNotPlanar);
    c->rejections++;
    return fail(MHD_INADMISSIBLE, "inadmissible cell average in a fixed-step sequence");
  }
  if (steps_done) *steps_done = nsteps;
  return MHD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Tile autotuner: elements per CTA of the volume kernel and of the magnetic
// stage kernels, timed on the context's own mesh and state.
// ---------------------------------------------------------------------------
namespace {

// Mean time of `reps` launches of fn() on the context stream (ms).
template <class F>
float time_launches(mhd_ctx* c, int reps, F fn, cudaEvent_t a, cudaEvent_t b) {
  fn();  // warm-up
  cudaEventRecord(a, c->st);
  for (int r = 0; r < reps; ++r) fn();
  cudaEventRecord(b, c->st);
  cudaEventSynchronize(b);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, a, b);
  return ms / reps;
}

}  // namespace

extern "C" {

int mhd_autotune(mhd_ctx* c, int* choices) {
  if (!c) return fail(MHD_EINVAL, "null context");
  const size_t N = c->N;
  const int reps = (int)std::min<long long>(100, std::max<long long>(3, 262144LL / c->M.K));
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return cuda_fail(e, "autotune events");
  set_scalar(c->dt, 0.0, c->st);  // tau = 0: the timed stages leave their inputs unchanged
  hydro_face(c->p, c->U, c->Fx, c->Fy, c->M, c->st);
  float best = 1e30f;
  int bv = 0;
  for (int v = 0; v < kTileVariants; ++v) {
    Mesh Mv = c->M;
    Mv.tile_vol = v;
    float t = time_launches(c, reps, [&] {
      hydro_vol(c->p, 1, c->U, c->U, c->Fx, c->Fy, c->S1, nullptr, c->status, c->T, Mv, c->dt, 1.0, 0.0, 1.0, 1,
                c->st);
    }, a, b);
    if (t < best) { best = t; bv = v; }
  }
  cons_to_prim(c->U, c->Y0, N, c->st);
  // magnetic stage: each kernel's own variant (tile code vE + 3 vJ + 9 vB), chosen
  // one kernel at a time with the others held: E (the largest) first, then J, then B
  int bv3[3] = {0, 0, 0};  // E, J, B
  for (int which = 0; which < 3; ++which) {
    best = 1e30f;
    int bw = 0;
    for (int v = 0; v < kTileVariants; ++v) {
      if (!mag_tile_ok(c->p, c->k, v)) continue;
      int trial[3] = {bv3[0], bv3[1], bv3[2]};
      trial[which] = v;
      Mesh Mv = c->M;
      Mv.tile_mag = trial[0] + kTileVariants * trial[1] + kTileVariants * kTileVariants * trial[2];
      float t = time_launches(c, reps, [&] {
        mag_stage(c->p, c->k, 0, c->B, c->Y0 + N, c->Y0, c->U, c->eta, 0, c->B, c->Y0 + N, c->Y0, c->Ba, c->Ya + N,
                  c->Ya, c->LJ, c->LE, c->T, Mv, c->dt, 1.0, 0.0, 1.0, 1, c->prm.reduced, c->st);
      }, a, b);
      if (t < best) { best = t; bw = v; }
    }
    bv3[which] = bw;
  }
  const int bm = bv3[0] + kTileVariants * bv3[1] + kTileVariants * kTileVariants * bv3[2];
  cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->st);
  e = cudaStreamSynchronize(c->st);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  c->M.tile_vol = bv;
  c->M.tile_mag = bm;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  if (choices) {
    choices[0] = vol_tile_eb(c->p, bv);
    choices[1] = mag_tile_eb(bv3[0]);
  }
  return MHD_OK;
}

int mhd_set_tiles(mhd_ctx* c, int vol_variant, int mag_variant) {
  if (!c) return fail(MHD_EINVAL, "null context");
  constexpr int V = kTileVariants;
  // one variant for the three magnetic kernels, or the code vE + 3 vJ + 9 vB
  const int code = mag_variant >= 0 && mag_variant < V ? mag_variant * (1 + V + V * V) : mag_variant;
  if (vol_variant < 0 || vol_variant >= V || code < 0 || code >= V * V * V || !mag_tile_ok(c->p, c->k, code % V) ||
      !mag_tile_ok(c->p, c->k, code / V % V) || !mag_tile_ok(c->p, c->k, code / (V * V)))
    return fail(MHD_EINVAL, "invalid tile variant");
  c->M.tile_vol = vol_variant;
  c->M.tile_mag = code;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return MHD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch of independent runs (uneven meshes and degrees): every run keeps its
// own context and stream; one CUDA graph holds a parallel branch per run, so a
// batch step is a single graph launch and small runs overlap on the GPU.
// ---------------------------------------------------------------------------
struct mhd_batch {
  std::vector<mhd_ctx*> runs;
  cudaStream_t root;
  std::vector<cudaEvent_t> ev;  // ev[0] fork, ev[1 + i] join of run i, ev[1 + n + i] set-up of run i
  cudaGraphExec_t exec;
  int exec_steps;
  long long launches_per_replay;
  long long launches_total;
  unsigned* h_status;
};

extern "C" {

int mhd_batch_create(int nruns, const mhd_mesh_t* meshes, const int* p, const int* k, const double* gamma,
                     mhd_batch** out) {
  if (!out || nruns < 1 || !meshes || !p || !k || !gamma) return fail(MHD_EINVAL, "invalid argument");
  *out = nullptr;
  mhd_batch* b = new (std::nothrow) mhd_batch();
  if (!b) return fail(MHD_ENOMEM, "host allocation");
  cudaError_t e = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete b; return cuda_fail(e, "stream"); }
  for (int i = 0; i < nruns; ++i) {
    mhd_ctx* c = nullptr;
    int r = mhd_create(&meshes[i], p[i], k[i], gamma[i], &c);
    if (r != MHD_OK) { mhd_batch_destroy(b); return r; }
    b->runs.push_back(c);
  }
  b->ev.resize(1 + 2 * nruns);
  for (auto& ev : b->ev)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
      mhd_batch_destroy(b);
      return cuda_fail(e, "events");
    }
  if ((e = cudaMallocHost(&b->h_status, sizeof(unsigned) * nruns)) != cudaSuccess) {
    mhd_batch_destroy(b);
    return cuda_fail(e, "pinned status");
  }
  *out = b;
  return MHD_OK;
}

void mhd_batch_destroy(mhd_batch* b) {
  if (!b) return;
  if (b->root) cudaStreamSynchronize(b->root);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto ev : b->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto c : b->runs) mhd_destroy(c);
  if (b->h_status) cudaFreeHost(b->h_status);
  if (b->root) cudaStreamDestroy(b->root);
  delete b;
}

int mhd_batch_size(const mhd_batch* b) { return b ? (int)b->runs.size() : 0; }

mhd_ctx* mhd_batch_run(mhd_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->runs.size()) return nullptr;
  return b->runs[i];
}

int mhd_batch_autotune(mhd_batch* b) {
  if (!b) return fail(MHD_EINVAL, "null batch");
  for (auto c : b->runs) {
    int r = mhd_autotune(c, nullptr);
    if (r != MHD_OK) return r;
  }
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  return MHD_OK;
}

int mhd_batch_step(mhd_batch* b, const double* dt, int nsteps, int* status) {
  if (!b || !dt || nsteps < 1) return fail(MHD_EINVAL, "invalid argument");
  const int n = (int)b->runs.size();
  for (int i = 0; i < n; ++i)
    if (!(dt[i] > 0)) return fail(MHD_EINVAL, "dt must be positive");
  cudaError_t e;
  // (re)capture the batch graph: fork from the root stream into every run's stream
  bool stale = !b->exec || b->exec_steps != nsteps;
  for (auto c : b->runs) stale = stale || !c->graph || c->graph_steps != nsteps;
  if (stale) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    for (auto c : b->runs) {  // per-run graphs also serve as the validity marker of the parameters
      int r = sequence_graph(c, nsteps);
      if (r != MHD_OK) return r;
    }
    cudaGraph_t g = nullptr;
    std::vector<long long> l0(n);
    for (int i = 0; i < n; ++i) l0[i] = b->runs[i]->launches;
    if ((e = cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e, "begin capture");
    cudaEventRecord(b->ev[0], b->root);
    for (int i = 0; i < n; ++i) {
      mhd_ctx* c = b->runs[i];
      cudaStreamWaitEvent(c->st, b->ev[0], 0);
      enqueue_sequence(c, nsteps);
      cudaEventRecord(b->ev[1 + i], c->st);
      cudaStreamWaitEvent(b->root, b->ev[1 + i], 0);
    }
    e = cudaStreamEndCapture(b->root, &g);
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->exec = nullptr; return cuda_fail(e, "graph instantiate"); }
    b->launches_per_replay = 0;
    for (int i = 0; i < n; ++i) {  // captured launches count at replay, not at capture
      b->launches_per_replay += b->runs[i]->launches - l0[i];
      b->runs[i]->launches = l0[i];
    }
    b->exec_steps = nsteps;
  }
  // per-run step length and status words, then the graph on the root stream
  for (int i = 0; i < n; ++i) {
    mhd_ctx* c = b->runs[i];
    cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->st);
    set_scalar(c->dt, dt[i], c->st);
    c->launches++;
    cudaEventRecord(b->ev[1 + n + i], c->st);
    cudaStreamWaitEvent(b->root, b->ev[1 + n + i], 0);
  }
  if ((e = cudaGraphLaunch(b->exec, b->root)) != cudaSuccess) return cuda_fail(e, "graph launch");
  b->launches_total += b->launches_per_replay;
  for (int i = 0; i < n; ++i)
    if ((e = cudaMemcpyAsync(&b->h_status[i], b->runs[i]->status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             b->root)) != cudaSuccess)
      return cuda_fail(e, "status copy");
  if ((e = cudaStreamSynchronize(b->root)) != cudaSuccess) return cuda_fail(e, "batch step");
  int worst = MHD_OK;
  for (int i = 0; i < n; ++i) {
    mhd_ctx* c = b->runs[i];
    int st = MHD_OK;
    if (b->h_status[i] & (ST_INADMISSIBLE | ST_NOT_PLANAR)) {  // restore this run; the caller may retry it
      cudaMemcpyAsync(c->U, c->Usave, 5 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      cudaMemcpyAsync(c->B, c->Bsave, 3 * c->Z * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
      cudaStreamSynchronize(c->st);
      st = (b->h_status[i] & ST_NOT_PLANAR) ? MHD_EINVAL : MHD_INADMISSIBLE;
      if (worst == MHD_OK || st == MHD_EINVAL) worst = st;
    }
    if (status) status[i] = st;
  }
  if (worst == MHD_EINVAL) return fail(worst, kNotPlanar);
  return worst == MHD_OK ? MHD_OK : fail(worst, "a run of the batch had an inadmissible cell average");
}

long long mhd_batch_launch_count(const mhd_batch* b) {
  if (!b) return 0;
  long long t = b->launches_total;
  for (auto c : b->runs) t += c->launches;
  return t;
}

int mhd_substep(mhd_ctx* c, int which, double tau) {
  if (!c || !(tau > 0) || (which != 0 && which != 1)) return fail(MHD_EINVAL, "invalid argument");
  cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->st);
  if (which == 1 && c->prm.reduced) {  // refuse before any change of the state
    unsigned s0 = 0;
    check_planar(c->U + 3 * c->N, c->N, c->B + 2 * c->Z, c->Z, c->status, c->st);
    int r0 = check_status(c, &s0);
    if (r0 != MHD_OK) return r0;
    if (s0 & ST_NOT_PLANAR) return fail(MHD_EINVAL, kNotPlanar);
  }
  set_scalar(c->dt, tau, c->st);
  c->launches++;
  if (which == 0) hydro_substep(c, 1.0);
  else mag_substep(c, 1.0);
  unsigned s = 0;
  int r = check_status(c, &s);
  if (r != MHD_OK) return r;
  if (s & ST_INADMISSIBLE) return fail(MHD_INADMISSIBLE, "inadmissible raw cell average");
  return MHD_OK;
}

int mhd_hydro_rhs(mhd_ctx* c, const double* U, double* L, int on_device) {
  if (!c || !U || !L) return fail(MHD_EINVAL, "null argument");
  cudaError_t e;
  if ((e = copy_in(c, c->S1, U, 5 * c->N, on_device)) != cudaSuccess) return cuda_fail(e, "U");
  hydro_face(c->p, c->S1, c->Fx, c->Fy, c->M, c->st);
  hydro_vol(c->p, 0, c->S1, c->S1, c->Fx, c->Fy, c->S2, nullptr, c->status, c->T, c->M, c->dt, 0.0, 0.0, 0.0, 0,
            c->st);
  c->launches += 2;
  if ((e = copy_out(c, L, c->S2, 5 * c->N, on_device)) != cudaSuccess) return cuda_fail(e, "L");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "hydro_rhs");
  return MHD_OK;
}

int mhd_hydro_stage_map(mhd_ctx* c, const double* U, double tau, double* out, int on_device) {
  if (!c || !U || !out) return fail(MHD_EINVAL, "null argument");
  if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(MHD_EINVAL, "tau must be finite and >= 0");
  cudaError_t e;
  if ((e = copy_in(c, c->S1, U, 5 * c->N, on_device)) != cudaSuccess) return cuda_fail(e, "U");
  cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->st);
  set_scalar(c->dt, tau, c->st);
  stab_hydro(c->p, c->S1, c->status, c->T, c->M, c->prm, c->dt, 1.0, c->work, nullptr, c->st);
  c->launches += 1 + (c->prm.oe_hydro ? kStatsLaunches + 1 : 1);
  if ((e = copy_out(c, out, c->S1, 5 * c->N, on_device)) != cudaSuccess) return cuda_fail(e, "out");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "hydro_stage_map");
  return MHD_OK;
}

int mhd_mag_rhs(mhd_ctx* c, const double* rho, const double* e_, const double* u, const double* Bx, const double* By,
                const double* Bz, const double* eta, double* de, double* du, double* dBx, double* dBy, double* dBz,
                int on_device) {
  if (!c || !rho || !e_ || !u || !Bx || !By || !Bz || !eta || !de || !du || !dBx || !dBy || !dBz)
    return fail(MHD_EINVAL, "null argument");
  const size_t N = c->N, Z = c->Z;
  cudaError_t e;
  // rho -> S1[0:N]; Y = [e | u] -> Ya; B -> Ba (blocked); eta -> work
  if ((e = copy_in(c, c->S1, rho, N, on_device)) != cudaSuccess) return cuda_fail(e, "rho");
  if ((e = copy_in(c, c->Ya, e_, N, on_device)) != cudaSuccess) return cuda_fail(e, "e");
  if ((e = copy_in(c, c->Ya + N, u, 3 * N, on_device)) != cudaSuccess) return cuda_fail(e, "u");
  if ((e = copy_in(c, c->io, Bx, Z, on_device)) != cudaSuccess) return cuda_fail(e, "Bx");
  grid_to_blocked(c->io, c->Ba, c->M.nx, c->M.ny, c->mm, c->st);
  if ((e = copy_in(c, c->io, By, Z, on_device)) != cudaSuccess) return cuda_fail(e, "By");
  grid_to_blocked(c->io, c->Ba + Z, c->M.nx, c->M.ny, c->mm, c->st);
  if ((e = copy_in(c, c->Ba + 2 * Z, Bz, Z, on_device)) != cudaSuccess) return cuda_fail(e, "Bz");
  if ((e = copy_in(c, c->work, eta, c->M.K, on_device)) != cudaSuccess) return cuda_fail(e, "eta");
  mag_stage(c->p, c->k, 0, c->Ba, c->Ya + N, c->Ya, c->S1, c->work, 1, c->Ba, c->Ya + N, c->Ya, c->Bb, c->Yb + N,
            c->Yb, c->LJ, c->LE, c->T, c->M, c->dt, 0.0, 0.0, 0.0, 0, 0, c->st);
  c->launches += 5;
  if ((e = copy_out(c, de, c->Yb, N, on_device)) != cudaSuccess) return cuda_fail(e, "de");
  if ((e = copy_out(c, du, c->Yb + N, 3 * N, on_device)) != cudaSuccess) return cuda_fail(e, "du");
  blocked_to_grid(c->Bb, c->io, c->M.nx, c->M.ny, c->mm, c->st);
  if ((e = copy_out(c, dBx, c->io, Z, on_device)) != cudaSuccess) return cuda_fail(e, "dBx");
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "dBx");
  blocked_to_grid(c->Bb + Z, c->io, c->M.nx, c->M.ny, c->mm, c->st);
  if ((e = copy_out(c, dBy, c->io, Z, on_device)) != cudaSuccess) return cuda_fail(e, "dBy");
  if ((e = copy_out(c, dBz, c->Bb + 2 * Z, Z, on_device)) != cudaSuccess) return cuda_fail(e, "dBz");
  c->launches += 2;
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(e, "mag_rhs");
  return MHD_OK;
}

int mhd_diagnostics(mhd_ctx* c, mhd_diag_t* out) {
  if (!c || !out) return fail(MHD_EINVAL, "null argument");
  const size_t K = c->M.K;
  diag_partials(c->p, c->k, c->U, c->B, c->T, c->M, c->work, c->st);
  c->launches++;
  std::vector<double> h(12 * K), eta(K);
  cudaError_t e = cudaMemcpyAsync(h.data(), c->work, 12 * K * sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(eta.data(), c->eta, K * sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_status + 1, c->prm.activity, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->prm.activity, 0, sizeof(unsigned), c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics");
  double acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1e300, 1e300};
  const int nx = c->M.nx;
  // a walled context reports its physical elements only (the images repeat them)
  auto physical = [&](size_t k) {
    return !c->walls || ((int)(k % nx) < c->pnx && (int)(k / nx) < c->pny);
  };
  for (size_t k = 0; k < K; ++k) {
    if (!physical(k)) continue;
    for (int q = 0; q < 8; ++q) acc[q] += h[k * 12 + q];
    acc[8] = std::max(acc[8], h[k * 12 + 8]);
    acc[9] = std::max(acc[9], h[k * 12 + 9]);
    acc[10] = std::min(acc[10], h[k * 12 + 10]);
    acc[11] = std::min(acc[11], h[k * 12 + 11]);
  }
  double emax = 0.0;
  for (size_t k = 0; k < K; ++k)
    if (physical(k)) emax = std::max(emax, eta[k]);
  out->mass = acc[0]; out->mom[0] = acc[1]; out->mom[1] = acc[2]; out->mom[2] = acc[3];
  out->E_kin = acc[4]; out->E_int = acc[5]; out->entropy = acc[6]; out->E_mag = 0.5 * acc[7];
  out->div_B = acc[8]; out->B_max = acc[9]; out->rho_min = acc[10]; out->p_min = acc[11];
  out->eta_max = emax;
  out->n_rejections = (int)c->rejections;
  out->stab_active = (int)c->h_status[1];
  return MHD_OK;
}

int mhd_get_eta(mhd_ctx* c, double* eta) {
  if (!c || !eta) return fail(MHD_EINVAL, "null argument");
  cudaError_t e = copy_out(c, eta, c->eta, c->M.K, 0);
  if (e != cudaSuccess) return cuda_fail(e, "get_eta");
  return MHD_OK;
}

long long mhd_launch_count(const mhd_ctx* c) { return c ? c->launches : 0; }

int mhd_profile_kernels(mhd_ctx* c, int enable) {
  if (!c) return fail(MHD_EINVAL, "null context");
  cudaStreamSynchronize(c->st);
  c->profiling = enable != 0;
  c->ev_rec.clear();
  return MHD_OK;
}

int mhd_kernel_times(mhd_ctx* c, double* ms, long long* counts, int nclasses) {
  if (!c || !ms || !counts) return fail(MHD_EINVAL, "null argument");
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel_times");
  for (int i = 0; i < nclasses; ++i) { ms[i] = 0.0; counts[i] = 0; }
  for (auto& r : c->ev_rec) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.second.first, r.second.second) != cudaSuccess) continue;
    if (r.first < nclasses) { ms[r.first] += t; counts[r.first]++; }
  }
  return KC_COUNT;
}

}  // extern "C"
