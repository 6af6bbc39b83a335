// Device random numbers shared by the CUDA sources: the counter-based Philox
// generator every draw is keyed on, and the rounded-normal table draw.
#pragma once
#include <cstdint>

#include "pulda_internal.h"

namespace pulda {

struct U4 { uint32_t x, y, z, w; };

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// Counter (a, b, sweep, tag << 28 | aux), key = the 64-bit seed.
__device__ __forceinline__ U4 draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t sweep, uint32_t tag, uint32_t aux) {
    return philox(a, b, sweep, (tag << 28) | (aux & 0x0FFFFFFFu), static_cast<uint32_t>(seed),
                  static_cast<uint32_t>(seed >> 32));
}

// A standard normal draw: one of 2^16 equiprobable cells of the normal law
// (x0's high 16 bits), linear inside the cell with a 48-bit position.
__device__ __forceinline__ double gauss_draw(const DevTables &T, uint32_t x0, uint32_t x1) {
    const uint32_t cell = x0 >> 16;
    const uint64_t frac48 = (static_cast<uint64_t>(x0 & 0xFFFFu) << 32) | x1;
    const double f = __dmul_rn(static_cast<double>(frac48), 3.552713678800501e-15);   // 2^-48
    const double a = T.gauss[cell], b = T.gauss[cell + 1];
    return __dadd_rn(a, __dmul_rn(__dsub_rn(b, a), f));
}

}  // namespace pulda
