#include "common.cuh"
namespace mbir {
bool wavelet_supported(int nx, int nz) { return nx % 8 == 0 && nz % 8 == 0 && nx / 4 >= 8 && nz / 4 >= 8; }
}
extern "C" {
int mbir_prox(mbir_plan, int32_t, const void*, double, void*, void*) { return MBIR_ERR_UNSUPPORTED_SIZE; }
int mbir_wavelet(mbir_plan, int32_t, const void*, void*, void*) { return MBIR_ERR_UNSUPPORTED_SIZE; }
}
