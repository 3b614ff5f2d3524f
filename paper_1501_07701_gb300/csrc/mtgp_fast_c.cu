// Instantiations of the register-resident kernel for M = ceil(N/32) in {44}
// (state sizes of the common MTGP32 exponents; see mtgp_fast.cuh).
#include "mtgp_fast.cuh"

namespace mtgp {

const void* fast_ptr_group_c(int M, int K)
{
    switch (M * 16 + K) {
    case 44 * 16 + 4: return (const void*)mtgp_fast_kernel<44, 4>;
    case 44 * 16 + 8: return (const void*)mtgp_fast_kernel<44, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
