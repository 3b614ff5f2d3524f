// Instantiations of the fused generation + statistics kernel for
// M = ceil(N/32) in {4, 5, 22, 23, 44} and G = 8 warps per CTA (see mtgp_fused.cuh).
#include "mtgp_fused.cuh"

namespace mtgp {

const void* fused_ptr_group_b(int M, int G)
{
    switch (M * 16 + G) {
    case 4 * 16 + 8: return (const void*)mtgp_fused_kernel<4, 8>;
    case 5 * 16 + 8: return (const void*)mtgp_fused_kernel<5, 8>;
    case 22 * 16 + 8: return (const void*)mtgp_fused_kernel<22, 8>;
    case 23 * 16 + 8: return (const void*)mtgp_fused_kernel<23, 8>;
    case 44 * 16 + 8: return (const void*)mtgp_fused_kernel<44, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
