// bap_fit.cuh -- declarations of the device kernels around the path kernel (bap_fit.cu).
#pragma once

#include "bap_internal.cuh"

namespace bap {

__global__ void korobov_merit_kernel(int J, int s, double* merit);
__global__ void korobov_pick_kernel(int J, int s, const double* merit, int* out_a);
__global__ void iz_setup_kernel(const DevModel* M, int m, int J, int n_bnd, const int* korobov_a,
                                double* start, ItemState* state, int* pivot, int* active,
                                int* count, const double* coef64, int n_coef, int degree,
                                const int* fitted, int warm_start, float* l0f);
__global__ void newton_items_setup_kernel(const DevModel* M, int m, int n_items, int n_bnd,
                                          const double* starts_in, const int* pivots_in,
                                          const int* ctr_in, double* start, ItemState* state,
                                          int* pivot, int* ctr_item, int* live_flag,
                                          const double* coef64, int n_coef, int degree,
                                          const int* fitted, int warm_start, float* l0f);
__global__ void newton_items_list_kernel(const int* live_flag, int n_items, int* active, int* count);
__global__ void stage_iz_kernel(const double* coef64, int n_dates, int n_bnd, int n_coef, int s,
                                int degree, double K, float* coef_f, double* coef_d);
// Threads per block of ls_fit_kernel (one block per boundary).
constexpr int kLsThreads = 256;
__global__ void ls_fit_kernel(const DevModel* M, int m, int J, int n_bnd, int degree, int n_coef,
                              const double* start, const ItemState* state, double* coef64,
                              float* coef_f, double* coef_d, int* fitted);
__global__ void train_points_kernel(const DevModel* M, int m, RoundKeys rk, int J, double* start,
                                    int* ctr_item, double* W, int bridge_from_next);
__global__ void stage_cmc_kernel(int n_dates, int nF, int max_stumps, const int* n_stumps,
                                 const int* feat, const double* thr, const int* pol,
                                 const double* alpha, int rec_len, float* rec_f, double* rec_d);
__global__ void adaboost_kernel(const DevModel* M, int m, int J, const double* X,
                                const double* label_y, const int* label, int n_rounds,
                                double* sorted_v, int* sorted_i, double* err, int max_stumps,
                                int* n_stumps, int* feat, double* thr, int* pol, double* alpha,
                                int rec_len, float* rec_f, double* rec_d, int* fitted);
// Threads per block of the cluster boosting kernels (one block per feature).
constexpr int kClusterBoostThreads = 1024;
__global__ void adaboost_cluster_kernel(const DevModel* M, int m, int J, const double* X,
                                        const int* label, int n_rounds, double* sorted_v,
                                        int* sorted_i, int max_stumps, int* n_stumps, int* feat,
                                        double* thr, int* pol, double* alpha, int rec_len,
                                        float* rec_f, double* rec_d, int* fitted);
// One-block AdaBoost with one warp per feature: threads per block, and the dynamic shared memory
// for J points and nF features (the sort region, later the FP64 and signed fixed-point weights;
// the 16-bit sorted orders in blocks of 1024 positions; three 64-bit values per segment of 32;
// the labels).
constexpr int kWarpBoostThreads = 512;
// Largest J for which the default boosting form picks the warp-per-feature block over the
// cluster (measured on GB300: the block is faster at J = 1024, the cluster at J = 4000).
constexpr int kWarpBoostAutoMaxJ = 2048;
__host__ __device__ inline size_t warp_boost_region(int J) {
    int P2 = 1;
    while (P2 < J) P2 <<= 1;
    const size_t a = (size_t)P2 * 12, b = (size_t)J * 16 + 8;
    return ((a > b ? a : b) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t warp_boost_smem(int J, int nF) {
    const size_t nsc = (size_t)(J + 1023) / 1024;
    return warp_boost_region(J) + (size_t)nF * nsc * 1024 * 2 + 3 * (size_t)nF * nsc * 32 * 8 +
           (size_t)J;
}
__global__ void adaboost_warp_kernel(const DevModel* M, int m, int J, const double* X,
                                     const int* label, int n_rounds, double* sorted_v,
                                     int* sorted_i, int max_stumps, int* n_stumps, int* feat,
                                     double* thr, int* pol, double* alpha, int rec_len,
                                     float* rec_f, double* rec_d, int* fitted);
__global__ void logitboost_cluster_kernel(const DevModel* M, int m, int J, const double* X,
                                          const int* label, int n_rounds, double* sorted_v,
                                          int* sorted_i, int max_stumps, int* n_stumps, int* feat,
                                          double* thr, int* pol, double* alpha, int rec_len,
                                          float* rec_f, double* rec_d, int* fitted);
__global__ void newton_decide_kernel(IterState* s, const int* count, int max_iter,
                                     cudaGraphConditionalHandle h, int* passes);
__global__ void set_int_kernel(int* p, int v);
__global__ void rng_debug_kernel(RoundKeys rk, uint32_t w1, uint32_t step, int d, long long count,
                                 uint32_t* words, double* z);
__global__ void collect_points_kernel(const ItemState* state, int n, double* x_out, int* it_out,
                                      int* st_out, int* counts);
__global__ void collect_labels_kernel(const double* label_y, int n, double* x_out, int* it_out,
                                      int* st_out);

// The path kernel of d = D for a rule (or kernel selector), FP32 or FP64, with ppl path slots per
// lane (2 exists for the FP32 quadratic I&Z kernels; otherwise the ppl = 1 kernel is returned),
// specialised for the payoff where such a kernel exists (payoff < 0: the general kernel).
template <int D> const void* path_kernel_fn(int rule, bool fp64, int ppl, int payoff);

}  // namespace bap
