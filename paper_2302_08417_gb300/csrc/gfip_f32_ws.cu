// FP32 GEMM on the warp-specialised tile core (gfip_ws.cuh): the launch every dense FP32
// GEMM of the library takes (fused, direct and pack-then-compute alike).
#include "gfip_ws.cuh"

namespace gfip {

cudaError_t launch_ws_gemm(const GemmParams<float> &p, cudaStream_t s)
{
    if (p.a_contig_m)
        return p.b_contig_n ? ws::launch_t<true, true>(p, s) : ws::launch_t<true, false>(p, s);
    return p.b_contig_n ? ws::launch_t<false, true>(p, s) : ws::launch_t<false, false>(p, s);
}

cudaError_t launch_ws_pack(const PackParams<float> &p, cudaStream_t s)
{
    if (p.a_contig_m)
        return p.b_contig_n ? ws::launch_pack_t<true, true>(p, s)
                            : ws::launch_pack_t<true, false>(p, s);
    return p.b_contig_n ? ws::launch_pack_t<false, true>(p, s)
                        : ws::launch_pack_t<false, false>(p, s);
}

int ws_blocks_per_sm()
{
    int n = ws::blocks_per_sm_one<true, true>();
    n = std::min(n, ws::blocks_per_sm_one<true, false>());
    n = std::min(n, ws::blocks_per_sm_one<false, true>());
    n = std::min(n, ws::blocks_per_sm_one<false, false>());
    return n;
}

}  // namespace gfip
