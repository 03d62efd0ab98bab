// Internal store helpers of the library kernels: 32-byte (256-bit) and
// 16-byte vector stores to global memory; CS = true uses the streaming
// (evict-first) cache policy.
#pragma once

#include <cstdint>

namespace sq {

template <bool CS>
__device__ __forceinline__ void store32B(void *p, const uint32_t (&v)[8]) {
    if constexpr (CS) {
        asm volatile("st.global.cs.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v[0]),
                     "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                     : "memory");
    } else {
        asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v[0]),
                     "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                     : "memory");
    }
}

template <bool CS>
__device__ __forceinline__ void store16B(void *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    if constexpr (CS) {
        asm volatile("st.global.cs.v4.b32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
                     "r"(d)
                     : "memory");
    } else {
        asm volatile("st.global.v4.b32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
                     "r"(d)
                     : "memory");
    }
}

}  // namespace sq
