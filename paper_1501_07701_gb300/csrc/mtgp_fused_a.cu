// Instantiations of the fused generation + statistics kernel for
// M = ceil(N/32) in {10, 11, 20} and G = 8 warps per CTA, with the dispatch and
// the launcher of every instantiation (see mtgp_fused.cuh).
#include "mtgp_fused.cuh"

namespace mtgp {

const void* fused_ptr_group_b(int M, int G);

static const void* fused_ptr_group_a(int M, int G)
{
    switch (M * 16 + G) {
    case 10 * 16 + 8: return (const void*)mtgp_fused_kernel<10, 8>;
    case 11 * 16 + 8: return (const void*)mtgp_fused_kernel<11, 8>;
    case 20 * 16 + 8: return (const void*)mtgp_fused_kernel<20, 8>;
    default: return nullptr;
    }
}

const void* fused_kernel_ptr(int M, int G)
{
    const void* p = fused_ptr_group_a(M, G);
    return p ? p : fused_ptr_group_b(M, G);
}

cudaError_t launch_fused(const void* fn, const GenArgs& a, const StatsArgs& A, dim3 grid, dim3 block,
                         size_t smem, cudaStream_t s)
{
    KParams P = a.P;
    uint32_t* states = a.states;
    uint32_t n_streams = a.n_streams;
    const WorkItem* items = a.items;
    const Segment* segs = a.segs;
    uint32_t n_items = a.n_items;
    uint32_t* counter = a.counter;
    uint32_t* out = a.out;
    int* err = a.err;
    const KSet* sets = a.sets;
    const uint32_t* set_of = a.set_of;
    StatsArgs st = A;
    void* args[] = {&P, &states, &n_streams, &items, &segs, &n_items, &counter, &out, &err,
                    &sets, &set_of, &st};
    return cudaLaunchKernel(fn, grid, block, args, smem, s);
}

}  // namespace mtgp
