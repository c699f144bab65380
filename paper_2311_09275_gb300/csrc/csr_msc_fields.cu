// csr_msc_fields.cu -- the multi-spin-coded colour-class sweep kernels with
// local fields (kernels in csr_msc.cuh), in a translation unit of their own
// so that the two sets of builds compile in parallel.
#include "csr_msc.cuh"

namespace isg {

cudaError_t gm_launch_fields(const GraphMscSolve &s, const GraphMscLaunch &l,
                             cudaStream_t stream) {
  return gm_launch_impl<true>(s, l, stream);
}

}  // namespace isg
