// Instantiations of the register-resident kernel for M = ceil(N/32) in {20,22,23}
// (state sizes of the common MTGP32 exponents; see mtgp_fast.cuh), for
// K sub-steps per parallel step and G warps per CTA.
#include "mtgp_fast.cuh"

namespace mtgp {

const void* fast_ptr_group_b(int M, int K, int G)
{
    switch ((M * 16 + K) * 16 + G) {
    case (20 * 16 + 8) * 16 + 2: return (const void*)mtgp_fast_kernel<20, 8, 2>;
    case (20 * 16 + 8) * 16 + 4: return (const void*)mtgp_fast_kernel<20, 8, 4>;
    case (20 * 16 + 8) * 16 + 8: return (const void*)mtgp_fast_kernel<20, 8, 8>;
    case (20 * 16 + 4) * 16 + 2: return (const void*)mtgp_fast_kernel<20, 4, 2>;
    case (20 * 16 + 4) * 16 + 4: return (const void*)mtgp_fast_kernel<20, 4, 4>;
    case (20 * 16 + 4) * 16 + 8: return (const void*)mtgp_fast_kernel<20, 4, 8>;
    case (22 * 16 + 8) * 16 + 2: return (const void*)mtgp_fast_kernel<22, 8, 2>;
    case (22 * 16 + 8) * 16 + 4: return (const void*)mtgp_fast_kernel<22, 8, 4>;
    case (22 * 16 + 8) * 16 + 8: return (const void*)mtgp_fast_kernel<22, 8, 8>;
    case (22 * 16 + 4) * 16 + 2: return (const void*)mtgp_fast_kernel<22, 4, 2>;
    case (22 * 16 + 4) * 16 + 4: return (const void*)mtgp_fast_kernel<22, 4, 4>;
    case (22 * 16 + 4) * 16 + 8: return (const void*)mtgp_fast_kernel<22, 4, 8>;
    case (23 * 16 + 8) * 16 + 2: return (const void*)mtgp_fast_kernel<23, 8, 2>;
    case (23 * 16 + 8) * 16 + 4: return (const void*)mtgp_fast_kernel<23, 8, 4>;
    case (23 * 16 + 8) * 16 + 8: return (const void*)mtgp_fast_kernel<23, 8, 8>;
    case (23 * 16 + 4) * 16 + 2: return (const void*)mtgp_fast_kernel<23, 4, 2>;
    case (23 * 16 + 4) * 16 + 4: return (const void*)mtgp_fast_kernel<23, 4, 4>;
    case (23 * 16 + 4) * 16 + 8: return (const void*)mtgp_fast_kernel<23, 4, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
