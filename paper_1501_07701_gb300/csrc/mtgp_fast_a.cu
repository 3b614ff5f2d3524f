// Instantiations of the register-resident kernel for M = ceil(N/32) in {10,11}
// (state sizes of the common MTGP32 exponents; see mtgp_fast.cuh).
#include "mtgp_fast.cuh"

namespace mtgp {

const void* fast_ptr_group_a(int M, int K)
{
    switch (M * 16 + K) {
    case 10 * 16 + 4: return (const void*)mtgp_fast_kernel<10, 4>;
    case 10 * 16 + 8: return (const void*)mtgp_fast_kernel<10, 8>;
    case 11 * 16 + 4: return (const void*)mtgp_fast_kernel<11, 4>;
    case 11 * 16 + 8: return (const void*)mtgp_fast_kernel<11, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
