// Instantiations of the register-resident kernel for M = ceil(N/32) in {10,11}
// (state sizes of the common MTGP32 exponents; see mtgp_fast.cuh), for
// K sub-steps per parallel step and G warps per CTA.
#include "mtgp_fast.cuh"

namespace mtgp {

const void* fast_ptr_group_a(int M, int K, int G)
{
    switch ((M * 16 + K) * 16 + G) {
    case (10 * 16 + 8) * 16 + 2: return (const void*)mtgp_fast_kernel<10, 8, 2>;
    case (10 * 16 + 8) * 16 + 4: return (const void*)mtgp_fast_kernel<10, 8, 4>;
    case (10 * 16 + 8) * 16 + 8: return (const void*)mtgp_fast_kernel<10, 8, 8>;
    case (10 * 16 + 4) * 16 + 2: return (const void*)mtgp_fast_kernel<10, 4, 2>;
    case (10 * 16 + 4) * 16 + 4: return (const void*)mtgp_fast_kernel<10, 4, 4>;
    case (10 * 16 + 4) * 16 + 8: return (const void*)mtgp_fast_kernel<10, 4, 8>;
    case (11 * 16 + 8) * 16 + 2: return (const void*)mtgp_fast_kernel<11, 8, 2>;
    case (11 * 16 + 8) * 16 + 4: return (const void*)mtgp_fast_kernel<11, 8, 4>;
    case (11 * 16 + 8) * 16 + 8: return (const void*)mtgp_fast_kernel<11, 8, 8>;
    case (11 * 16 + 4) * 16 + 2: return (const void*)mtgp_fast_kernel<11, 4, 2>;
    case (11 * 16 + 4) * 16 + 4: return (const void*)mtgp_fast_kernel<11, 4, 4>;
    case (11 * 16 + 4) * 16 + 8: return (const void*)mtgp_fast_kernel<11, 4, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
