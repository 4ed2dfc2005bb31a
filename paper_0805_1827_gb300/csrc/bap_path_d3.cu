// Path kernels for d = 3 (one translation unit per d, so that nvcc works on them in parallel).
#include "bap_path_inst.inc"
namespace bap {
template const void* path_kernel_fn<3>(int, bool, int, int);
}
