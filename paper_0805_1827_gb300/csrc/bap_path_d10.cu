// Path kernels for d = 10 (one translation unit per d, so that nvcc works on them in parallel).
#include "bap_path_inst.inc"
namespace bap {
template const void* path_kernel_fn<10>(int, bool, int, int);
}
