// Philox4x32-10 words from PyTorch's host-side engine (ATen's
// PhiloxRNGEngine.h, an implementation of Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11, written by a third
// party).  The tests call it as an independent library routine to pin the
// oracle's generator, which is written separately from the same definition.
//
// The engine's state maps onto the generator's 128-bit counter and 64-bit
// key as: key = seed (low word first), counter words 2-3 = subsequence,
// counter words 0-1 = offset; each call returns the next of the four words
// of the current block, word 0 first.
#include <ATen/core/PhiloxRNGEngine.h>

#include <cstdint>

extern "C" void library_philox4x32_10(int64_t n, const uint32_t* ctr /* n x 4 */,
                                      const uint32_t* key /* n x 2 */, uint32_t* out /* n x 4 */) {
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t* c = ctr + 4 * i;
        const uint32_t* k = key + 2 * i;
        at::philox_engine e(uint64_t(k[0]) | (uint64_t(k[1]) << 32),
                            uint64_t(c[2]) | (uint64_t(c[3]) << 32),
                            uint64_t(c[0]) | (uint64_t(c[1]) << 32));
        for (int w = 0; w < 4; ++w) out[4 * i + w] = e();
    }
}
