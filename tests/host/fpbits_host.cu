// Host build of the bit-pattern conversions of the multigrid's level-0 casts (fpbits.cuh).
#include "../../paper_0908_2654_gb300/csrc/fpbits.cuh"

extern "C" {
void to_float_scaled_host(int n, const double* v, int e, float* out) {
    for (int i = 0; i < n; ++i) out[i] = fpbits::to_float_scaled(v[i], e);
}
void from_float_scaled_host(int n, const float* v, int e, double* out) {
    for (int i = 0; i < n; ++i) out[i] = fpbits::from_float_scaled(v[i], e);
}
void pow2_exponent_host(int n, const double* v, int* out) {
    for (int i = 0; i < n; ++i) out[i] = fpbits::pow2_exponent(v[i]);
}
}
