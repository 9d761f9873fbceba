// k_gate_bh_fwd.cu -- block gate kernels: forward application, Bose-Hubbard fixed-N sector.
#include "k_gate_impl.cuh"

namespace cvq {

template void launch_block<CVQ_BH, false>(const SectorDev&, const GateArg&, PoolDev, const cdf*, cdf*, cdf*, double*, size_t,
                                     cudaStream_t);
template void set_block_smem_limit<CVQ_BH, false>(int);

}  // namespace cvq
