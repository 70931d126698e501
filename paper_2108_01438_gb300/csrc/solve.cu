#include "common.cuh"
namespace mbir {
void destroy_solve_state(mbir_plan) {}
}
extern "C" {
int mbir_solve(mbir_plan, const void*, const uint8_t*, const mbir_solve_opts*, void*, mbir_solve_info*, void*) {
  return MBIR_ERR_UNSUPPORTED_SIZE;
}
int mbir_lipschitz(mbir_plan, const uint8_t*, int32_t, double*, void*) { return MBIR_ERR_UNSUPPORTED_SIZE; }
}
