// Ragged batches: argument checks only until the persistent kernel lands.
#include "../../include/gb300fft.h"
#include "fft_internal.h"

extern "C" {
fft_plan_t fft_plan_create_ragged(int count, const int *nx, const int *ny, int dir, int precision) {
    auto pow2_in = [](int n) { return n >= 32 && n <= 1024 && (n & (n - 1)) == 0; };
    if (count < 1 || !nx || !ny) {
        gb300fft::set_last_error(count < 1 ? FFT_ERR_INVALID_SIZE : FFT_ERR_INVALID_ARG);
        return nullptr;
    }
    for (int i = 0; i < count; ++i)
        if (!pow2_in(nx[i]) || !pow2_in(ny[i])) {
            gb300fft::set_last_error(FFT_ERR_INVALID_SIZE);
            return nullptr;
        }
    (void)dir;
    (void)precision;
    gb300fft::set_last_error(FFT_ERR_UNSUPPORTED);
    return nullptr;
}
int fft_ragged_offset(fft_plan_t, int, long long *) { return FFT_ERR_INVALID_ARG; }
int fft_execute_ragged(fft_plan_t, const void *, void *, void *) { return FFT_ERR_UNSUPPORTED; }
int fft_execute_ragged_loop(fft_plan_t, const void *, void *, void *) { return FFT_ERR_UNSUPPORTED; }
}
