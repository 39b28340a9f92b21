// Compile-time loop: calls f(std::integral_constant<int, I>) for I in [B, E).
#pragma once

#include <type_traits>

namespace lbm {

template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

}  // namespace lbm
