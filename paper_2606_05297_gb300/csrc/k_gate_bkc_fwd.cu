// k_gate_bkc_fwd.cu -- block gate kernels: forward application, Kitaev-chain parity sector.
#include "k_gate_impl.cuh"

namespace cvq {

template void launch_block<CVQ_BKC, false>(const SectorDev&, const GateArg&, PoolDev, const cdf*, cdf*, cdf*, double*, size_t,
                                     cudaStream_t);
template void set_block_smem_limit<CVQ_BKC, false>(int);

}  // namespace cvq
