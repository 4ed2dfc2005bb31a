// Path kernels for d = 1..3.
#include "bap_path_inst.inc"
namespace bap {
template const void* path_kernel_fn<1>(int, bool, int, int);
template const void* path_kernel_fn<2>(int, bool, int, int);
template const void* path_kernel_fn<3>(int, bool, int, int);
}
