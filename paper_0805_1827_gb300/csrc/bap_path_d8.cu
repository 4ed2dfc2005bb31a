// Path kernels for d = 8..10.
#include "bap_path_inst.inc"
namespace bap {
template const void* path_kernel_fn<8>(int, bool, int, int);
template const void* path_kernel_fn<9>(int, bool, int, int);
template const void* path_kernel_fn<10>(int, bool, int, int);
}
