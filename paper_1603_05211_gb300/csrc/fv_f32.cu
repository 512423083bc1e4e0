// Finite-volume stage and CFL kernels instantiated for float state.
#include "fv_inst.cuh"
namespace mrfv {
MRFV_INSTANTIATE_FV(float)
}
