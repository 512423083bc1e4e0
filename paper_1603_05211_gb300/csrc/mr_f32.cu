// Multiresolution kernels instantiated for float state.
#include "mr_inst.cuh"
namespace mrfv {
MRFV_INSTANTIATE_MR(float)
}
