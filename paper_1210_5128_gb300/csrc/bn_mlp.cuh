// bn_mlp.cuh -- device state of the learned swap proposal (bn_mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include "bn_internal.cuh"

struct bn_mlp {
    int n = 0, d = 0, H = 0, P = 0, Pp = 0, nd = 0, ndp = 0, cap = 0, Mp = 0;
    float lr = 0.f, beta1 = 0.9f, beta2 = 0.999f, adam_eps = 1e-8f;
    int64_t t = 0;                 // Adam steps taken
    void* block = nullptr;
    size_t bytes = 0;
    // FP32 master weights (W1 padded to H x ndp, W3 to Pp x H), gradients, Adam moments
    float *E, *W1, *b1, *W2, *b2, *W3, *b3;
    float *gE, *gW1, *gb1, *gW2, *gb2, *gW3, *gb3;
    float *mE, *mW1, *mb1, *mW2, *mb2, *mW3, *mb3;
    float *vE, *vW1, *vb1, *vW2, *vb2, *vW3, *vb3;
    // bf16 GEMM operands
    __nv_bfloat16 *Eb, *W1b, *W1T, *W2b, *W2T, *W3b;
    __nv_bfloat16 *X, *XT, *H1, *H1T, *H2, *dZ2, *dZ2T, *dZ1, *dZ1T;
    // FP32 activations
    float *Z1, *Z2, *L, *dH1, *dX, *loss;
    float *grow, *lrow;            // per training row: d loss / d logit[pair] and loss term
    uint8_t* inv = nullptr;        // [cap][64] inverse orders of a training batch
    float* ws = nullptr;           // split-K partials
    size_t ws_elems = 0;
    uint32_t* status;
    uint8_t* stage_orders;
    uint32_t* stage_pairs;
    float* stage_alpha;
};

namespace bn {
int gemm_tc(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc, int M, int N,
            int K, uint32_t* status, cudaStream_t s, float* ws, size_t ws_elems);
// forward of B orders (device pointer); logits land in m->L (row stride Pp)
int mlp_forward_dev(bn_mlp* m, const uint8_t* d_orders, int B, bool keep_transposes, cudaStream_t s);
int mlp_loss_grad_dev(bn_mlp* m, const uint8_t* d_orders, const uint32_t* d_pairs, const float* d_alpha, int B,
                      cudaStream_t s);
int mlp_adam_dev(bn_mlp* m, cudaStream_t s);
}  // namespace bn
