// Stage stabilisation kernels (hydro OE + positivity limiter, A.R.
// coefficient, velocity OE).  Not built yet: the API rejects enabling them.
#include "mhd_internal.cuh"

namespace mhd {
void stab_hydro(int, double*, const double*, unsigned*, const Tab*, const Mesh&, const Stab&, const double*, double,
                double*, cudaStream_t) {}
void stab_eta(int, int, const double*, const double*, const double*, const Tab*, const Mesh&, const Stab&, double*,
              double*, cudaStream_t) {}
void stab_vel_prep(int, const double*, double*, const Tab*, const Mesh&, cudaStream_t) {}
void stab_vel(int, int, const double*, double*, const double*, const double*, const Tab*, const Mesh&, const Stab&,
              const double*, double, double*, cudaStream_t) {}
size_t stab_work_doubles(int, int, const Mesh& M) { return 16 * (size_t)M.K; }
size_t stab_chol_doubles(int, const Mesh&) { return 1; }
}  // namespace mhd
