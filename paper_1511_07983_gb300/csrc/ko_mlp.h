// Surrogate MLP: sizes, parameter layout and kernel launchers (ko_mlp.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ko_internal.h"

constexpr int kSlots = 24;        // position slots
constexpr int kSlotFeat = 7;      // features per slot
constexpr int kGlobals = 8;       // global features
constexpr int kMlpIn = 192;       // 24*7 + 8 = 176, padded to 192
constexpr int kHidden = 256;
constexpr int kMaxK = KO_MAX_KERNELS;

constexpr int kEpiReluBf16 = 0;
constexpr int kEpiF32 = 1;

// Flat FP32 parameter layout: W1 [192 x 256] (k-major), b1 [256], W2 [256 x 256],
// b2, W3 [256 x 256], b3, w4 [256], b4 [1].
constexpr long long kOffW1 = 0;
constexpr long long kOffB1 = kOffW1 + (long long)kMlpIn * kHidden;
constexpr long long kOffW2 = kOffB1 + kHidden;
constexpr long long kOffB2 = kOffW2 + (long long)kHidden * kHidden;
constexpr long long kOffW3 = kOffB2 + kHidden;
constexpr long long kOffB3 = kOffW3 + (long long)kHidden * kHidden;
constexpr long long kOffW4 = kOffB3 + kHidden;
constexpr long long kOffB4 = kOffW4 + kHidden;
constexpr long long kParams = kOffB4 + 1;

cudaError_t ko_mlp_gemm_relu(const uint16_t *A, int lda, const uint16_t *Bt, int ldb, int M, int N, int K,
                             const float *bias, uint16_t *out, int ldo, uint16_t *out_t, int ldt,
                             cudaStream_t st);
// tcgen05 forward layer: out = bf16(relu(A Wt^T + bias)), M % 128 == 0,
// K in {192, 256}, N = 256; *err set to 1 if the MMA completion wait gave up.
cudaError_t ko_mlp_layer_tc(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                            int *err, cudaStream_t st);
// tcgen05 last hidden layer fused with the output layer: y = a . w4 + b4 with
// a = bf16(relu(A Wt^T + bias)) (not stored), in ko_mlp_out_fwd's summation
// order, so y has the same bits as ko_mlp_layer_tc followed by
// ko_mlp_out_fwd (which is what runs, through `out`, when the fused kernel
// does not fit).  Same shapes as ko_mlp_layer_tc.
cudaError_t ko_mlp_layer_tc_out(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias,
                                const uint16_t *w4, const float *b4, uint16_t *out, float *y, int *err,
                                cudaStream_t st);
// tcgen05 training forward layer: also writes out_t = out transposed
// ([256][ldt] BF16, ldt % 8 == 0).  Same shapes as ko_mlp_layer_tc.
cudaError_t ko_mlp_layer_tc_t(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                              uint16_t *out_t, long long ldt, int *err, cudaStream_t st);
// tcgen05 input gradient: outf[M][256] = A Wt^T in FP32 (M % 128 == 0, K in {192, 256}).
cudaError_t ko_mlp_layer_tc_f32(const uint16_t *A, const uint16_t *Wt, int M, int K, float *outf, int *err,
                                cudaStream_t st);
// tcgen05 weight gradient: out[M][256] (row stride ldo) = A Bt^T with
// A [M][Kdim] (row stride lda), Bt [256][Kdim] (row stride ldb), M <= 256,
// Kdim % 256 == 0; split-K over 256-wide slices into `work`
// (ko_mlp_wgrad_tc_workspace bytes), summed in a fixed order.
size_t ko_mlp_wgrad_tc_workspace(int M, long long Kdim);
cudaError_t ko_mlp_wgrad_tc(const uint16_t *A, long long lda, const uint16_t *Bt, long long ldb, int M,
                            long long Kdim, float *out, int ldo, float *work, int *err, cudaStream_t st);
cudaError_t ko_mlp_gemm_f32(const uint16_t *A, int lda, const uint16_t *Bt, int ldb, int M, int N, int K,
                            float *out, int ldo, cudaStream_t st);
cudaError_t ko_mlp_encode(const int8_t *rows, int row_stride, const int *sid, const int *pick,
                          const int *set_n, const float *kfeat, const float *gfeat, int B, uint16_t *x,
                          uint16_t *xt, cudaStream_t st);
cudaError_t ko_mlp_out_fwd(const uint16_t *a3, const uint16_t *w4, const float *b4, int B, float *y,
                           cudaStream_t st);
// The backward kernels sum per-block partials (workspace `part`, at least
// ko_mlp_part_floats(B) floats) in a fixed order: gradients are reproducible.
size_t ko_mlp_part_floats(int B);
cudaError_t ko_mlp_out_bwd(const float *y, const float *t, const uint16_t *a3, const uint16_t *w4, int B,
                           float *loss_sum, float *dw4, float *db4, float *db3, uint16_t *dz,
                           uint16_t *dzt, float *part, cudaStream_t st);
cudaError_t ko_mlp_relu_bwd(const float *da, const uint16_t *a, int B, float *db, uint16_t *dz,
                            uint16_t *dzt, float *part, cudaStream_t st);
cudaError_t ko_mlp_adam(float *p, float *m, float *v, const float *g, long long count, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st);
cudaError_t ko_mlp_weights_bf16(const float *w, int K, int N, uint16_t *wk, uint16_t *wt, cudaStream_t st);
cudaError_t ko_mlp_topk(const float *y, long long n, int k, uint32_t *state, unsigned int *hist,
                        unsigned int *counters, int *out, cudaStream_t st);
cudaError_t ko_mlp_random_orders(int8_t *rows, int stride, long long count, int n, unsigned long long seed,
                                 cudaStream_t st);
cudaError_t ko_mlp_targets(const int64_t *ms, const int *sid, const double *log2_lb, long long n, float *t,
                           cudaStream_t st);
cudaError_t ko_mlp_pick(int *pick, int B, long long pool, unsigned long long seed, const float *t_src,
                        float *t_dst, cudaStream_t st);
cudaError_t ko_mlp_neighbours(const int8_t *base, int beam, int n, int8_t *out, cudaStream_t st);
cudaError_t ko_mlp_gather_rows(const int8_t *src, int stride, const int *pick, int B, int8_t *dst,
                               cudaStream_t st);
