// Instantiations of the register-resident kernel for M = ceil(N/32) in {44}
// (state sizes of the common MTGP32 exponents; see mtgp_fast.cuh), for
// K sub-steps per parallel step and G warps per CTA.
#include "mtgp_fast.cuh"

namespace mtgp {

const void* fast_ptr_group_c(int M, int K, int G)
{
    switch ((M * 16 + K) * 16 + G) {
    case (44 * 16 + 8) * 16 + 2: return (const void*)mtgp_fast_kernel<44, 8, 2>;
    case (44 * 16 + 8) * 16 + 4: return (const void*)mtgp_fast_kernel<44, 8, 4>;
    case (44 * 16 + 8) * 16 + 8: return (const void*)mtgp_fast_kernel<44, 8, 8>;
    case (44 * 16 + 4) * 16 + 2: return (const void*)mtgp_fast_kernel<44, 4, 2>;
    case (44 * 16 + 4) * 16 + 4: return (const void*)mtgp_fast_kernel<44, 4, 4>;
    case (44 * 16 + 4) * 16 + 8: return (const void*)mtgp_fast_kernel<44, 4, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
