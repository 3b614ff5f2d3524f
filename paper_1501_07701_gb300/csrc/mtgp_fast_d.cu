// Instantiations of the register-resident kernel for short states:
// M = ceil(N/32) in {4, 5} (Mexp 3217, the exponent of the paper's 10 000
// statuses, and 4253 / 4423), for K sub-steps per parallel step and G warps
// per CTA.  Seed-generated Mexp 3217 sets have N - pos between 64 and 99, so
// they take K = 2 (64-word steps).
#include "mtgp_fast.cuh"

namespace mtgp {

const void* fast_ptr_group_d(int M, int K, int G)
{
    switch ((M * 16 + K) * 16 + G) {
    case (4 * 16 + 2) * 16 + 2: return (const void*)mtgp_fast_kernel<4, 2, 2>;
    case (4 * 16 + 2) * 16 + 4: return (const void*)mtgp_fast_kernel<4, 2, 4>;
    case (4 * 16 + 2) * 16 + 8: return (const void*)mtgp_fast_kernel<4, 2, 8>;
    case (5 * 16 + 2) * 16 + 2: return (const void*)mtgp_fast_kernel<5, 2, 2>;
    case (5 * 16 + 2) * 16 + 4: return (const void*)mtgp_fast_kernel<5, 2, 4>;
    case (5 * 16 + 2) * 16 + 8: return (const void*)mtgp_fast_kernel<5, 2, 8>;
    case (5 * 16 + 4) * 16 + 2: return (const void*)mtgp_fast_kernel<5, 4, 2>;
    case (5 * 16 + 4) * 16 + 4: return (const void*)mtgp_fast_kernel<5, 4, 4>;
    case (5 * 16 + 4) * 16 + 8: return (const void*)mtgp_fast_kernel<5, 4, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
