// k_gate_bkc_adj.cu -- block gate kernels: reverse (adjoint) step, Kitaev-chain parity sector.
#include "k_gate_impl.cuh"

namespace cvq {

template void launch_block<CVQ_BKC, true>(const SectorDev&, const GateArg&, PoolDev, const cdf*, cdf*, cdf*, double*, size_t,
                                     cudaStream_t);
template void set_block_smem_limit<CVQ_BKC, true>(int);

}  // namespace cvq
