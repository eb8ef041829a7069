// Host entry points of the D3Q19 path (called by the lbm_* dispatch).
#pragma once

#include <string>

#include "lbm.h"

namespace lbm3 {

struct Ctx3;

lbm_status create(const lbm_grid* g, const lbm_params* p, const lbm_open_bc* bcs, int nbc, const uint8_t* solid,
                  const double* rho_init, const double* u_init, void* stream, Ctx3** out, std::string* err);
void destroy(Ctx3* c);
const char* error(const Ctx3* c);
lbm_status reset(Ctx3* c, const double* rho_init, const double* u_init);
lbm_status step(Ctx3* c, int64_t nsteps);
lbm_status sync(Ctx3* c);
lbm_status enable_timing(Ctx3* c, int every);
lbm_status kernel_time_split(Ctx3* c, double* pull_ms, double* collide_ms, int64_t* samples);
lbm_status get_macros(Ctx3* c, float* rho, float* u, int dst_is_device);
lbm_status get_macros_f64(Ctx3* c, double* rho, double* u);
lbm_status get_populations(Ctx3* c, double* f);
lbm_status set_populations(Ctx3* c, const double* f);
lbm_status diagnostics(Ctx3* c, lbm_diag* d);

}  // namespace lbm3
