// Hydro residual without any device allocation: mhd_hydro_rhs_static().
//
// The ordinary entry points keep their scratch (the face fluxes among others)
// in memory that mhd_create() allocates.  Some callers cannot allocate device
// memory themselves: code that must run while all device memory belongs to a
// caching allocator or a fixed budget of the host application, or a latency-
// critical loop where a cudaMalloc/cudaFree pair is not acceptable.  For them
// this file offers the residual L_E of one conservative state with the face
// fluxes kept in a fixed, file-scope device array instead.
//
// The array is part of the library image: every GPU on which the library is
// used holds it (MHD_STATIC_SCRATCH_DOUBLES doubles, 8 MiB) until the process
// exits.  All calls share it, so calls whose kernels overlap on the GPU (two
// streams, two host threads) race on it; serialise them.  Every entry the
// residual reads is written by the same call first, so nothing in the array
// has to start at zero and stale contents from an earlier call are harmless.
#include <cstdio>

#include "../../include/mhd.h"
#include "mhd_internal.cuh"

namespace mhd {
void set_error_message(const char* msg);
void hydro_face(int p, const double* S, double* Fx, double* Fy, const Mesh& M, cudaStream_t st);
void hydro_vol(int p, int mode, const double* S, const double* U0, const double* Fx, const double* Fy, double* out,
               double* avg, unsigned* status, const Tab* T, const Mesh& M, const double* dtp, double dtfac,
               double ca, double cb, int first, cudaStream_t st);
}  // namespace mhd

#define MHD_STATIC_SCRATCH_DOUBLES (1u << 20)

// Face-flux scratch of the allocation-free residual (host code must not use
// this name as an address: it is a host-side stand-in for the device array).
static __device__ __align__(256) double g_static_scratch[MHD_STATIC_SCRATCH_DOUBLES];

namespace {
thread_local char g_static_err[256];

int static_fail(int code) {
  mhd::set_error_message(g_static_err);
  return code;
}

// Device address of g_static_scratch in the current context.  Looked up on
// every call (a cheap runtime query): a cached address would dangle after
// cudaDeviceReset() or in a new primary context.
double* static_scratch_ptr(int* code) {
  double* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    snprintf(g_static_err, sizeof g_static_err, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    *code = static_fail(MHD_ECUDA);
    return nullptr;
  }
  *code = MHD_OK;
  return p;
}
}  // namespace

extern "C" int mhd_hydro_rhs_static(const mhd_mesh_t* mesh, int p, double gamma, const double* U, double* L,
                                    void* stream) {
  if (!mesh || !U || !L) {
    snprintf(g_static_err, sizeof g_static_err, "null argument");
    return static_fail(MHD_EINVAL);
  }
  if (p < 1 || p > 4 || mesh->nx < 1 || mesh->ny < 1 || !(mesh->x1 > mesh->x0) || !(mesh->y1 > mesh->y0) ||
      !(gamma > 1.0)) {
    snprintf(g_static_err, sizeof g_static_err, "invalid mesh, degree (1..4) or gamma");
    return static_fail(MHD_EINVAL);
  }
  const unsigned long long K = (unsigned long long)mesh->nx * (unsigned long long)mesh->ny;
  const unsigned long long need = 2ull * 5ull * K * (unsigned long long)(p + 1);  // x- and y-face fluxes
  if (need > MHD_STATIC_SCRATCH_DOUBLES) {
    snprintf(g_static_err, sizeof g_static_err,
             "mesh too large for the static scratch: needs %llu doubles (10 K (p+1)), limit %u", need,
             (unsigned)MHD_STATIC_SCRATCH_DOUBLES);
    return static_fail(MHD_EINVAL);
  }
  int code = MHD_OK;
  double* scratch = static_scratch_ptr(&code);
  if (!scratch) return code;
  cudaError_t e = cudaSuccess;
  // p is the magnetic degree too here: the residual does not touch the
  // magnetic tables, and (p, p) is always a supported pair.
  const mhd::Tab* T = mhd::device_tables(p, p, &e);
  if (!T) {
    snprintf(g_static_err, sizeof g_static_err, "tables: %s", cudaGetErrorString(e));
    return static_fail(MHD_ECUDA);
  }
  mhd::Mesh M{};  // default tile variants (0)
  M.nx = mesh->nx; M.ny = mesh->ny; M.K = (int)K;
  M.hx = (mesh->x1 - mesh->x0) / mesh->nx;
  M.hy = (mesh->y1 - mesh->y0) / mesh->ny;
  M.Jdet = M.hx * M.hy / 4.0;
  M.g = gamma;
  mhd::mesh_reciprocals(M);
  cudaStream_t st = (cudaStream_t)stream;
  double* Fx = scratch;
  double* Fy = scratch + 5ull * K * (p + 1);
  mhd::hydro_face(p, U, Fx, Fy, M, st);
  mhd::hydro_vol(p, 0, U, U, Fx, Fy, L, nullptr, nullptr, T, M, nullptr, 0.0, 0.0, 0.0, 0, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_static_err, sizeof g_static_err, "launch: %s", cudaGetErrorString(e));
    return static_fail(MHD_ECUDA);
  }
  return MHD_OK;
}
