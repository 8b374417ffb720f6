// Column-layout advisor (Algorithm 5).
#include "kernels.h"

extern "C" int bs_advise_layout(const int32_t *h_values, uint64_t n, int32_t mode, const bs_encode_opts *opts,
                                bs_advice *out) {
    (void)h_values; (void)n; (void)mode; (void)opts; (void)out;
    return BS_ERR_UNSUPPORTED;
}
