// Multiresolution kernels instantiated for double state.
#include "mr_inst.cuh"
namespace mrfv {
MRFV_INSTANTIATE_MR(double)
}
