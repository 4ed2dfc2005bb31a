// Path kernels for d = 4..5.
#include "bap_path_inst.inc"
namespace bap {
template const void* path_kernel_fn<4>(int, bool, int, int);
template const void* path_kernel_fn<5>(int, bool, int, int);
}
