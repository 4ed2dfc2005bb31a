// Path kernels for d = 6..7.
#include "bap_path_inst.inc"
namespace bap {
template const void* path_kernel_fn<6>(int, bool, int, int);
template const void* path_kernel_fn<7>(int, bool, int, int);
}
