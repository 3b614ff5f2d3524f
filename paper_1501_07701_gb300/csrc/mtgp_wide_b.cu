// Instantiations of the wide-column kernel (mtgp_wide.cuh) for NS = ceil(N/128)
// in {6, 11} (Mexp 21701, 23209 and 44497, and the literal 727 / 1392 rows)
// and G warps per CTA.
#include "mtgp_wide.cuh"

namespace mtgp {

const void* wide_ptr_group_b(int NS, int G)
{
    switch (NS * 16 + G) {
    case 6 * 16 + 4: return (const void*)mtgp_wide_kernel<6, 4>;
    case 6 * 16 + 8: return (const void*)mtgp_wide_kernel<6, 8>;
    case 11 * 16 + 4: return (const void*)mtgp_wide_kernel<11, 4>;
    case 11 * 16 + 8: return (const void*)mtgp_wide_kernel<11, 8>;
    default: return nullptr;
    }
}

}  // namespace mtgp
