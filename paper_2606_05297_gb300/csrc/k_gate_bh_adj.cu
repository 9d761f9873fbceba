// k_gate_bh_adj.cu -- block gate kernels: reverse (adjoint) step, Bose-Hubbard fixed-N sector.
#include "k_gate_impl.cuh"

namespace cvq {

template void launch_block<CVQ_BH, true>(const SectorDev&, const GateArg&, PoolDev, const cdf*, cdf*, cdf*, double*, size_t,
                                     cudaStream_t);
template void set_block_smem_limit<CVQ_BH, true>(int);

}  // namespace cvq
