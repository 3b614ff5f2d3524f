// Instantiations of the wide-column kernel (mtgp_wide.cuh) for NS = ceil(N/128)
// in {3, 4, 5} (Mexp 9689 .. 19937) and G warps per CTA, plus the lookup of
// every instantiation.
#include "mtgp_wide.cuh"

namespace mtgp {

const void* wide_ptr_group_b(int NS, int G);

const void* wide_kernel_ptr(int NS, int G)
{
    switch (NS * 16 + G) {
    case 3 * 16 + 4: return (const void*)mtgp_wide_kernel<3, 4>;
    case 3 * 16 + 8: return (const void*)mtgp_wide_kernel<3, 8>;
    case 4 * 16 + 4: return (const void*)mtgp_wide_kernel<4, 4>;
    case 4 * 16 + 8: return (const void*)mtgp_wide_kernel<4, 8>;
    case 5 * 16 + 4: return (const void*)mtgp_wide_kernel<5, 4>;
    case 5 * 16 + 8: return (const void*)mtgp_wide_kernel<5, 8>;
    default: return wide_ptr_group_b(NS, G);
    }
}

}  // namespace mtgp
