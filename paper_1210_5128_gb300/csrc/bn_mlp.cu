// bn_mlp.cu -- the learned swap proposal: a small MLP over the current order whose
// output is a distribution over the n(n-1)/2 swap pairs, used inside an exact MH ratio.
// The paper proposes uniform swaps (Sec. III.C); this network and its training target
// are the build's own specification (see include/bn.h).
//
// Dense layers run on the 5th-generation tensor cores: k_gemm_tc is a bf16 x bf16 -> f32
// GEMM, C = A B^T with both operands K-major, 128 x 128 tiles, a 3-stage cp.async
// pipeline into no-swizzle core-matrix shared-memory layouts, tcgen05.mma issued by one
// thread into a TMEM accumulator, completion through tcgen05.commit on an mbarrier, and
// a tcgen05.ld epilogue.  Bias, ReLU, bf16 rounding, transposed copies, the loss
// gradient, the scatter of the embedding gradient and Adam are small elementwise kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bn_tc.cuh"
#include "bn_mlp.cuh"

namespace bn {

typedef __nv_bfloat16 bf16;

static constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 3;
static constexpr int TC_TILE = TC_BM * TC_BK * 2;                       // bytes of one operand tile
static constexpr size_t TC_SMEM = 2 * TC_STAGES * TC_TILE + 256 + 1024;  // tiles + barriers + align slack
static constexpr uint32_t TC_IDESC = tc_idesc_bf16_f32(TC_BM, TC_BN);

struct GemmArgs {
    const bf16* A;   // M x K, row stride lda (elements)
    const bf16* B;   // N x K, row stride ldb
    float* C;        // M x N, row stride ldc; with split-K: partials [split][M][N]
    int M, N, K, lda, ldb, ldc;
    int ksplit;      // K / ksplit per CTA along grid z (1 = no split)
    uint32_t* status;
};

// core-matrix layout of a 128 x 64 bf16 tile: row r, 16-byte chunk kc of the row
__device__ __forceinline__ uint32_t tc_tile_off(int r, int kc) { return (r >> 3) * 1024 + kc * 128 + (r & 7) * 16; }

__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + TC_STAGES * TC_TILE;
    uint64_t* bar = (uint64_t*)(smem + 2 * TC_STAGES * TC_TILE);
    uint32_t* tslot = (uint32_t*)(bar + TC_STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
    const int kpart = g.K / g.ksplit;               // this CTA's K range (multiple of 64)
    const int kbase = blockIdx.z * kpart;
    const int nk = kpart / TC_BK;
    float* Cz = g.C + (size_t)blockIdx.z * g.M * g.ldc;

    if (warp == 0) {
        tc_alloc(tslot, 128);
        tc_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    auto load_stage = [&](int kt, int s) {
        uint8_t* a = sA + s * TC_TILE;
        uint8_t* b = sB + s * TC_TILE;
        for (int c = tid; c < TC_BM * 8; c += 128) {
            const int r = c >> 3, kc = c & 7;
            cp_async16(a + tc_tile_off(r, kc), g.A + (size_t)(m0 + r) * g.lda + kbase + kt * TC_BK + kc * 8);
            cp_async16(b + tc_tile_off(r, kc), g.B + (size_t)(n0 + r) * g.ldb + kbase + kt * TC_BK + kc * 8);
        }
        cp_async_commit();
    };

    for (int s = 0; s < TC_STAGES - 1; ++s) {
        if (s < nk) load_stage(s, s);
        else cp_async_commit();
    }
    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % TC_STAGES;
        const int kp = kt + TC_STAGES - 1;
        if (kp < nk) {
            const int sp = kp % TC_STAGES;        // last read by the MMAs of step kt-1
            if (kt >= 1) ok &= mbar_wait_bounded(&bar[sp], (uint32_t)(((kt - 1) / TC_STAGES) & 1), WAIT_TIMEOUT_NS);
            load_stage(kp, sp);
        } else {
            cp_async_commit();
        }
        cp_async_wait<TC_STAGES - 1>();            // step kt's tiles have landed
        fence_proxy_async_smem();                  // visible to the tensor core's async proxy
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t ad = tc_smem_desc(sA + s * TC_TILE + kk * 256, 128, 1024);
                const uint64_t bd = tc_smem_desc(sB + s * TC_TILE + kk * 256, 128, 1024);
                tc_mma_bf16(tmem, ad, bd, TC_IDESC, (kt > 0) || (kk > 0));
            }
            tc_commit(&bar[s]);
        }
    }
    if (nk > 0) ok &= mbar_wait_bounded(&bar[(nk - 1) % TC_STAGES], (uint32_t)(((nk - 1) / TC_STAGES) & 1),
                                        WAIT_TIMEOUT_NS);
    tc_fence_after();
    const bool all_ok = __syncthreads_and(ok);
    if (all_ok) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < TC_BN; c0 += 32) {
            uint32_t r[32];
            tc_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            tc_wait_ld();
            float* dst = Cz + (size_t)row * g.ldc + n0 + c0;
            if (nk > 0) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *(float4*)(dst + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                      __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
            } else {
#pragma unroll
                for (int j = 0; j < 32; j += 4) *(float4*)(dst + j) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    } else if (tid == 0) {
        atomicOr(g.status, STATUS_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 128);
}

// C = sum over the split partials, in split order (deterministic)
__global__ void k_splitk_reduce(const float* __restrict__ ws, int ksplit, int M, int N, float* __restrict__ C,
                                int ldc)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * N) return;
    const int r = (int)(idx / N), c = (int)(idx - (int64_t)r * N);
    float s = 0.f;
    for (int z = 0; z < ksplit; ++z) s += ws[(size_t)z * M * N + idx];
    C[(size_t)r * ldc + c] = s;
}

// C = A B^T.  Few output tiles and a long K split K over grid z (each CTA at least four
// 64-wide stages) into the workspace, then one reduction; ws == nullptr disables it.
int gemm_tc(const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M, int N, int K,
            uint32_t* status, cudaStream_t s, float* ws, size_t ws_elems)
{
    if (M % TC_BM || N % TC_BN || K % TC_BK)
        return set_error(BN_EINVAL, "gemm: M=%d N=%d K=%d must be multiples of 128, 128, 64", M, N, K);
    static unsigned long long ctx[64] = {0};
    if (first_in_context(ctx))
        BN_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    const int tiles = (M / TC_BM) * (N / TC_BN);
    int split = 1;
    if (ws) {
        const int stages = K / TC_BK;
        const int lim = std::min(sm_count() / std::max(tiles, 1), stages / 4);
        for (int dv = lim; dv >= 2; --dv)
            if (stages % dv == 0 && (size_t)dv * M * N <= ws_elems) {
                split = dv;
                break;
            }
    }
    GemmArgs g{A, B, split > 1 ? ws : C, M, N, K, lda, ldb, split > 1 ? N : ldc, split, status};
    k_gemm_tc<<<dim3(N / TC_BN, M / TC_BM, split), 128, TC_SMEM, s>>>(g);
    BN_LAUNCH_CHECK("k_gemm_tc");
    if (split > 1) {
        const int64_t tot = (int64_t)M * N;
        k_splitk_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ws, split, M, N, C, ldc);
        BN_LAUNCH_CHECK("k_splitk_reduce");
    }
    return BN_OK;
}

// ---------------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------------

// x rows: X[r][p*d + j] = E[order_r(p)][j] (bf16), zero padding; XT optional (transposed)
__global__ void k_embed(const uint8_t* __restrict__ orders, int B, int n, int d, int ndp, int Mp,
                        const bf16* __restrict__ Eb, bf16* __restrict__ X, bf16* __restrict__ XT)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Mp * ndp) return;
    const int r = (int)(idx / ndp), col = (int)(idx - (int64_t)r * ndp);
    bf16 v = __float2bfloat16_rn(0.f);
    if (r < B && col < n * d) {
        const int p = col / d, j = col - p * d;
        v = Eb[(size_t)orders[(size_t)r * n + p] * d + j];
    }
    X[idx] = v;
    if (XT) XT[(size_t)col * Mp + r] = v;
}

// Z += bias; H = bf16(relu(Z)) (rows >= B -> 0); HT optional
__global__ void k_bias_relu(float* __restrict__ Z, const float* __restrict__ bias, int Mp, int N, int B,
                            bf16* __restrict__ H, bf16* __restrict__ HT)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Mp * N) return;
    const int r = (int)(idx / N), c = (int)(idx - (int64_t)r * N);
    const float z = Z[idx] + bias[c];
    Z[idx] = z;
    const bf16 h = __float2bfloat16_rn(r < B ? fmaxf(z, 0.f) : 0.f);
    H[idx] = h;
    if (HT) HT[(size_t)c * Mp + r] = h;
}

__global__ void k_bias(float* __restrict__ Z, const float* __restrict__ bias, int Mp, int N)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Mp * N) return;
    Z[idx] += bias[idx % N];
}

// output layer gradient of the BCE loss (one logit per row): block per row.  The row's
// d loss / d logit and loss term go to grow[r] and lrow[r]; k_out_grad_w and k_loss_sum
// sum them in row order, so the gradients and the loss do not depend on scheduling.
__global__ void k_out_grad(const float* __restrict__ L, int ldl, const uint32_t* __restrict__ pairs,
                           const float* __restrict__ alpha, int B, int Mp, int H, const float* __restrict__ Z2,
                           const bf16* __restrict__ W3b, bf16* __restrict__ dZ2, bf16* __restrict__ dZ2T,
                           float* __restrict__ grow, float* __restrict__ lrow)
{
    const int r = blockIdx.x;
    float g = 0.f;
    int p = 0;
    if (r < B) {
        p = (int)pairs[r];
        const float l = L[(size_t)r * ldl + p];
        const float s = 1.f / (1.f + expf(-l));
        const float a = alpha[r];
        g = (s - a) / (float)B;
        if (threadIdx.x == 0) {
            lrow[r] = -(a * logf(s + 1e-30f) + (1.f - a) * logf(1.f - s + 1e-30f)) / (float)B;
            grow[r] = g;
        }
    }
    for (int c = threadIdx.x; c < H; c += blockDim.x) {
        bf16 dz = __float2bfloat16_rn(0.f);
        if (r < B) {
            const float dh = g * __bfloat162float(W3b[(size_t)p * H + c]);
            dz = __float2bfloat16_rn(Z2[(size_t)r * H + c] > 0.f ? dh : 0.f);
        }
        dZ2[(size_t)r * H + c] = dz;
        dZ2T[(size_t)c * Mp + r] = dz;
    }
}

// gW3 and gb3 rows of the pairs the batch touches: the block of the first row holding a
// pair sums that pair's rows in row order (the other rows of the pair leave it)
__global__ void k_out_grad_w(const uint32_t* __restrict__ pairs, const float* __restrict__ grow, int B, int H,
                             const bf16* __restrict__ H2, float* __restrict__ gW3, float* __restrict__ gb3)
{
    const int r = blockIdx.x;
    const uint32_t p = pairs[r];
    bool dup = false;
    for (int q = threadIdx.x; q < r; q += blockDim.x) dup |= pairs[q] == p;
    if (__syncthreads_or(dup)) return;                                  // block-uniform
    for (int c = threadIdx.x; c < H; c += blockDim.x) {
        float s = 0.f;
        for (int q = r; q < B; ++q)
            if (pairs[q] == p) s += grow[q] * __bfloat162float(H2[(size_t)q * H + c]);
        gW3[(size_t)p * H + c] = s;
    }
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int q = r; q < B; ++q)
            if (pairs[q] == p) s += grow[q];
        gb3[p] = s;
    }
}

// the batch loss: the rows' terms in a fixed order (per thread a strided run, then a
// fixed shared-memory tree)
__global__ void k_loss_sum(const float* __restrict__ lrow, int B, float* __restrict__ loss)
{
    __shared__ float red[256];
    float s = 0.f;
    for (int r = threadIdx.x; r < B; r += 256) s += lrow[r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0];
}

// dZ = bf16(dH * (Z > 0)), rows >= B -> 0, with the transposed copy
__global__ void k_relu_grad(const float* __restrict__ dH, const float* __restrict__ Z, int Mp, int N, int B,
                            bf16* __restrict__ dZ, bf16* __restrict__ dZT)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Mp * N) return;
    const int r = (int)(idx / N), c = (int)(idx - (int64_t)r * N);
    const bf16 v = __float2bfloat16_rn((r < B && Z[idx] > 0.f) ? dH[idx] : 0.f);
    dZ[idx] = v;
    dZT[(size_t)c * Mp + r] = v;
}

// column sums over the first B rows of a bf16 matrix (bias gradients)
__global__ void k_colsum(const bf16* __restrict__ M, int N, int B, float* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int r = 0; r < B; ++r) s += __bfloat162float(M[(size_t)r * N + c]);
    out[c] = s;
}

// inverse of each order: inv[r * 64 + v] = position of node v in order r
__global__ void k_inv_orders(const uint8_t* __restrict__ orders, int n, uint8_t* __restrict__ inv)
{
    const int r = blockIdx.x, p = threadIdx.x;
    if (p < n) inv[(size_t)r * 64 + orders[(size_t)r * n + p]] = (uint8_t)p;
}

// dE[v][j] = sum over the rows r, in row order, of dX[r][inv_r(v) d + j]
__global__ void k_embed_grad(const uint8_t* __restrict__ inv, const float* __restrict__ dX, int B, int n, int d,
                             int ndp, float* __restrict__ gE)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * d) return;
    const int v = idx / d, j = idx - v * d;
    float s = 0.f;
    for (int r = 0; r < B; ++r) s += dX[(size_t)r * ndp + (size_t)inv[(size_t)r * 64 + v] * d + j];
    gE[idx] = s;
}

// Adam (Kingma & Ba): moments and the FP32 master weight
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 copy of a rows x cols FP32 matrix (row stride ld), zero-padded to prow x pcol,
// and optionally its transpose (pcol x prow)
__global__ void k_to_bf16(const float* __restrict__ src, int ld, int rows, int cols, int prow, int pcol,
                          bf16* __restrict__ dst, bf16* __restrict__ dstT)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)prow * pcol) return;
    const int r = (int)(idx / pcol), c = (int)(idx - (int64_t)r * pcol);
    const bf16 v = __float2bfloat16_rn((r < rows && c < cols) ? src[(size_t)r * ld + c] : 0.f);
    if (dst) dst[idx] = v;
    if (dstT) dstT[(size_t)c * prow + r] = v;
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace bn

using namespace bn;

// ---------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------
static int mlp_refresh_bf16(bn_mlp* m, cudaStream_t s)
{
    k_to_bf16<<<nblk((int64_t)m->n * m->d), 256, 0, s>>>(m->E, m->d, m->n, m->d, m->n, m->d, m->Eb, nullptr);
    BN_LAUNCH_CHECK("k_to_bf16");
    k_to_bf16<<<nblk((int64_t)m->H * m->ndp), 256, 0, s>>>(m->W1, m->ndp, m->H, m->nd, m->H, m->ndp, m->W1b,
                                                          m->W1T);
    BN_LAUNCH_CHECK("k_to_bf16");
    k_to_bf16<<<nblk((int64_t)m->H * m->H), 256, 0, s>>>(m->W2, m->H, m->H, m->H, m->H, m->H, m->W2b, m->W2T);
    BN_LAUNCH_CHECK("k_to_bf16");
    k_to_bf16<<<nblk((int64_t)m->Pp * m->H), 256, 0, s>>>(m->W3, m->H, m->P, m->H, m->Pp, m->H, m->W3b, nullptr);
    BN_LAUNCH_CHECK("k_to_bf16");
    return BN_OK;
}

// forward of B <= cap orders already staged in m->orders_dev
int bn::mlp_forward_dev(bn_mlp* m, const uint8_t* d_orders, int B, bool keep_transposes, cudaStream_t s)
{
    const int Mp = (int)round_up(std::max(B, 1), 128);
    if (Mp > m->cap) return set_error(BN_EINVAL, "mlp: batch %d above capacity %d", B, m->cap);
    m->Mp = Mp;
    k_embed<<<nblk((int64_t)Mp * m->ndp), 256, 0, s>>>(d_orders, B, m->n, m->d, m->ndp, Mp, m->Eb, m->X,
                                                      keep_transposes ? m->XT : nullptr);
    BN_LAUNCH_CHECK("k_embed");
    int rc;
    if ((rc = gemm_tc(m->X, m->ndp, m->W1b, m->ndp, m->Z1, m->H, Mp, m->H, m->ndp, m->status, s, m->ws, m->ws_elems))) return rc;
    k_bias_relu<<<nblk((int64_t)Mp * m->H), 256, 0, s>>>(m->Z1, m->b1, Mp, m->H, B, m->H1,
                                                        keep_transposes ? m->H1T : nullptr);
    BN_LAUNCH_CHECK("k_bias_relu");
    if ((rc = gemm_tc(m->H1, m->H, m->W2b, m->H, m->Z2, m->H, Mp, m->H, m->H, m->status, s, m->ws, m->ws_elems))) return rc;
    k_bias_relu<<<nblk((int64_t)Mp * m->H), 256, 0, s>>>(m->Z2, m->b2, Mp, m->H, B, m->H2, nullptr);
    BN_LAUNCH_CHECK("k_bias_relu");
    if ((rc = gemm_tc(m->H2, m->H, m->W3b, m->H, m->L, m->Pp, Mp, m->Pp, m->H, m->status, s, m->ws, m->ws_elems))) return rc;
    k_bias<<<nblk((int64_t)Mp * m->Pp), 256, 0, s>>>(m->L, m->b3, Mp, m->Pp);
    BN_LAUNCH_CHECK("k_bias");
    return BN_OK;
}

int bn::mlp_loss_grad_dev(bn_mlp* m, const uint8_t* d_orders, const uint32_t* d_pairs, const float* d_alpha, int B,
                          cudaStream_t s)
{
    int rc = mlp_forward_dev(m, d_orders, B, true, s);
    if (rc) return rc;
    const int Mp = m->Mp, H = m->H;
    BN_CUDA(cudaMemsetAsync(m->gE, 0, sizeof(float) * (size_t)m->n * m->d, s));
    BN_CUDA(cudaMemsetAsync(m->gW3, 0, sizeof(float) * (size_t)m->P * H, s));
    BN_CUDA(cudaMemsetAsync(m->gb3, 0, sizeof(float) * (size_t)m->P, s));
    k_out_grad<<<Mp, 256, 0, s>>>(m->L, m->Pp, d_pairs, d_alpha, B, Mp, H, m->Z2, m->W3b, m->dZ2, m->dZ2T,
                                  m->grow, m->lrow);
    BN_LAUNCH_CHECK("k_out_grad");
    k_out_grad_w<<<B, 256, 0, s>>>(d_pairs, m->grow, B, H, m->H2, m->gW3, m->gb3);
    BN_LAUNCH_CHECK("k_out_grad_w");
    k_loss_sum<<<1, 256, 0, s>>>(m->lrow, B, m->loss);
    BN_LAUNCH_CHECK("k_loss_sum");
    k_colsum<<<nblk(H), 256, 0, s>>>(m->dZ2, H, B, m->gb2);
    BN_LAUNCH_CHECK("k_colsum");
    // dW2 = dZ2^T H1 ; dH1 = dZ2 W2
    if ((rc = gemm_tc(m->dZ2T, Mp, m->H1T, Mp, m->gW2, H, H, H, Mp, m->status, s, m->ws, m->ws_elems))) return rc;
    if ((rc = gemm_tc(m->dZ2, H, m->W2T, H, m->dH1, H, Mp, H, H, m->status, s, m->ws, m->ws_elems))) return rc;
    k_relu_grad<<<nblk((int64_t)Mp * H), 256, 0, s>>>(m->dH1, m->Z1, Mp, H, B, m->dZ1, m->dZ1T);
    BN_LAUNCH_CHECK("k_relu_grad");
    k_colsum<<<nblk(H), 256, 0, s>>>(m->dZ1, H, B, m->gb1);
    BN_LAUNCH_CHECK("k_colsum");
    // dW1 = dZ1^T X ; dX = dZ1 W1
    if ((rc = gemm_tc(m->dZ1T, Mp, m->XT, Mp, m->gW1, m->ndp, H, m->ndp, Mp, m->status, s, m->ws, m->ws_elems))) return rc;
    if ((rc = gemm_tc(m->dZ1, H, m->W1T, H, m->dX, m->ndp, Mp, m->ndp, H, m->status, s, m->ws, m->ws_elems))) return rc;
    k_inv_orders<<<B, 64, 0, s>>>(d_orders, m->n, m->inv);
    BN_LAUNCH_CHECK("k_inv_orders");
    k_embed_grad<<<nblk((int64_t)m->n * m->d), 256, 0, s>>>(m->inv, m->dX, B, m->n, m->d, m->ndp, m->gE);
    BN_LAUNCH_CHECK("k_embed_grad");
    return BN_OK;
}

int bn::mlp_adam_dev(bn_mlp* m, cudaStream_t s)
{
    m->t += 1;
    const float c1 = 1.f - powf(m->beta1, (float)m->t), c2 = 1.f - powf(m->beta2, (float)m->t);
    struct P {
        float *w, *g, *mm, *vv;
        int64_t cnt;
    } ps[7] = {{m->E, m->gE, m->mE, m->vE, (int64_t)m->n * m->d},
               {m->W1, m->gW1, m->mW1, m->vW1, (int64_t)m->H * m->ndp},
               {m->b1, m->gb1, m->mb1, m->vb1, (int64_t)m->H},
               {m->W2, m->gW2, m->mW2, m->vW2, (int64_t)m->H * m->H},
               {m->b2, m->gb2, m->mb2, m->vb2, (int64_t)m->H},
               {m->W3, m->gW3, m->mW3, m->vW3, (int64_t)m->P * m->H},
               {m->b3, m->gb3, m->mb3, m->vb3, (int64_t)m->P}};
    for (auto& p : ps) {
        k_adam<<<nblk(p.cnt), 256, 0, s>>>(p.w, p.g, p.mm, p.vv, p.cnt, m->lr, m->beta1, m->beta2, m->adam_eps, c1, c2);
        BN_LAUNCH_CHECK("k_adam");
    }
    return mlp_refresh_bf16(m, s);
}

extern "C" int bn_mlp_create(int n, const bn_mlp_params* p, const float* E, const float* W1, const float* b1,
                             const float* W2, const float* b2, const float* W3, const float* b3, int mem, void* stream,
                             bn_mlp** out)
{
    set_error(BN_OK, "");
    if (!out || !p) return set_error(BN_EINVAL, "bn_mlp_create: NULL argument");
    *out = nullptr;
    if (n < 2 || n > MAXN || p->d < 1 || p->hidden < 128 || p->hidden % 128 || p->batch_cap < 1 ||
        !(p->lr >= 0.f))
        return set_error(BN_EINVAL, "bn_mlp_create: bad sizes (hidden must be a positive multiple of 128)");
    if (!E || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return set_error(BN_EINVAL, "bn_mlp_create: NULL weights");
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_mlp_create: bad mem");
    cudaStream_t s = (cudaStream_t)stream;
    bn_mlp* m = new bn_mlp();
    m->n = n;
    m->d = p->d;
    m->H = p->hidden;
    m->P = n * (n - 1) / 2;
    m->Pp = (int)round_up(m->P, 128);
    m->nd = n * p->d;
    m->ndp = (int)round_up(m->nd, 128);
    m->cap = (int)round_up(p->batch_cap, 128);
    m->lr = p->lr;
    m->beta1 = p->beta1 > 0 ? p->beta1 : 0.9f;
    m->beta2 = p->beta2 > 0 ? p->beta2 : 0.999f;
    m->adam_eps = p->adam_eps > 0 ? p->adam_eps : 1e-8f;
    const int H = m->H, ndp = m->ndp, Pp = m->Pp, cap = m->cap;
    const size_t nE = (size_t)n * m->d, nW1 = (size_t)H * ndp, nW2 = (size_t)H * H, nW3 = (size_t)Pp * H;
    // one FP32 block: master (E W1 b1 W2 b2 W3 b3) x {w, grad, m, v}, activations
    size_t off = 0;
    std::vector<std::pair<float**, size_t>> f32 = {
        {&m->E, nE}, {&m->W1, nW1}, {&m->b1, (size_t)H}, {&m->W2, nW2}, {&m->b2, (size_t)H}, {&m->W3, nW3},
        {&m->b3, (size_t)Pp}, {&m->gE, nE}, {&m->gW1, nW1}, {&m->gb1, (size_t)H}, {&m->gW2, nW2},
        {&m->gb2, (size_t)H}, {&m->gW3, nW3}, {&m->gb3, (size_t)Pp}, {&m->mE, nE}, {&m->mW1, nW1},
        {&m->mb1, (size_t)H}, {&m->mW2, nW2}, {&m->mb2, (size_t)H}, {&m->mW3, nW3}, {&m->mb3, (size_t)Pp},
        {&m->vE, nE}, {&m->vW1, nW1}, {&m->vb1, (size_t)H}, {&m->vW2, nW2}, {&m->vb2, (size_t)H},
        {&m->vW3, nW3}, {&m->vb3, (size_t)Pp}, {&m->Z1, (size_t)cap * H}, {&m->Z2, (size_t)cap * H},
        {&m->L, (size_t)cap * Pp}, {&m->dH1, (size_t)cap * H}, {&m->dX, (size_t)cap * ndp}, {&m->loss, 4},
        {&m->grow, (size_t)cap}, {&m->lrow, (size_t)cap},
        {&m->ws, (size_t)8 * cap * std::max(std::max(Pp, ndp), H)}};
    std::vector<std::pair<bf16**, size_t>> b16 = {
        {&m->Eb, nE}, {&m->W1b, nW1}, {&m->W1T, nW1}, {&m->W2b, nW2}, {&m->W2T, nW2}, {&m->W3b, nW3},
        {&m->X, (size_t)cap * ndp}, {&m->XT, (size_t)cap * ndp}, {&m->H1, (size_t)cap * H},
        {&m->H1T, (size_t)cap * H}, {&m->H2, (size_t)cap * H}, {&m->dZ2, (size_t)cap * H},
        {&m->dZ2T, (size_t)cap * H}, {&m->dZ1, (size_t)cap * H}, {&m->dZ1T, (size_t)cap * H}};
    std::vector<size_t> offs;
    for (auto& e : f32) { offs.push_back(off); off = (size_t)round_up((int64_t)(off + 4 * e.second), 256); }
    for (auto& e : b16) { offs.push_back(off); off = (size_t)round_up((int64_t)(off + 2 * e.second), 256); }
    const size_t o_status = off;
    off += 256;
    const size_t o_stage = off;                      // staging for host inputs: orders, pairs, alpha
    off += (size_t)round_up((int64_t)cap * n, 256) + (size_t)round_up((int64_t)cap * 4, 256) * 2;
    const size_t o_inv = off;                        // inverse orders of a training batch
    off += (size_t)round_up((int64_t)cap * 64, 256);
    cudaError_t e = cudaMalloc(&m->block, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return set_error(BN_ENOMEM, "bn_mlp_create: %zu bytes: %s", off, cudaGetErrorString(e));
    }
    uint8_t* base = (uint8_t*)m->block;
    size_t k = 0;
    for (auto& e2 : f32) *e2.first = (float*)(base + offs[k++]);
    for (auto& e2 : b16) *e2.first = (bf16*)(base + offs[k++]);
    m->status = (uint32_t*)(base + o_status);
    m->stage_orders = base + o_stage;
    m->stage_pairs = (uint32_t*)(base + o_stage + (size_t)round_up((int64_t)cap * n, 256));
    m->stage_alpha = (float*)((uint8_t*)m->stage_pairs + (size_t)round_up((int64_t)cap * 4, 256));
    m->inv = base + o_inv;
    m->bytes = off;
    m->ws_elems = (size_t)8 * cap * std::max(std::max(Pp, ndp), H);
    auto fail = [&](int rc) { bn_mlp_free(m); return rc; };
    if (cudaMemsetAsync(m->block, 0, off, s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__));
    const cudaMemcpyKind kind = mem == BN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // weights come row-major and unpadded: E n x d, W1 H x (n d), W2 H x H, W3 P x H
    if (cudaMemcpyAsync(m->E, E, 4 * nE, kind, s) != cudaSuccess ||
        cudaMemcpy2DAsync(m->W1, 4 * (size_t)ndp, W1, 4 * (size_t)m->nd, 4 * (size_t)m->nd, H, kind, s) != cudaSuccess ||
        cudaMemcpyAsync(m->b1, b1, 4 * (size_t)H, kind, s) != cudaSuccess ||
        cudaMemcpyAsync(m->W2, W2, 4 * nW2, kind, s) != cudaSuccess ||
        cudaMemcpyAsync(m->b2, b2, 4 * (size_t)H, kind, s) != cudaSuccess ||
        cudaMemcpyAsync(m->W3, W3, 4 * (size_t)m->P * H, kind, s) != cudaSuccess ||
        cudaMemcpyAsync(m->b3, b3, 4 * (size_t)m->P, kind, s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "bn_mlp_create weights", __FILE__, __LINE__));
    int rc = mlp_refresh_bf16(m, s);
    if (rc) return fail(rc);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "sync", __FILE__, __LINE__));
    *out = m;
    return BN_OK;
}

static int stage_in(void* dst, const void* src, size_t bytes, int mem, cudaStream_t s, const void** out)
{
    if (mem == BN_MEM_DEVICE) { *out = src; return BN_OK; }
    BN_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    *out = dst;
    return BN_OK;
}

static int check_status(bn_mlp* m, cudaStream_t s, const char* who)
{
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, m->status, 4, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "%s: a bounded device wait expired", who);
    return BN_OK;
}

extern "C" int bn_mlp_forward(bn_mlp* m, const uint8_t* orders, int B, float* logits, int mem, void* stream)
{
    set_error(BN_OK, "");
    if (!m || !orders || !logits || B < 1) return set_error(BN_EINVAL, "bn_mlp_forward: bad arguments");
    if (B > m->cap) return set_error(BN_EINVAL, "bn_mlp_forward: B=%d above batch capacity %d", B, m->cap);
    cudaStream_t s = (cudaStream_t)stream;
    const void* d_o = nullptr;
    int rc = stage_in(m->stage_orders, orders, (size_t)B * m->n, mem, s, &d_o);
    if (rc) return rc;
    if ((rc = mlp_forward_dev(m, (const uint8_t*)d_o, B, false, s))) return rc;
    BN_CUDA(cudaMemcpy2DAsync(logits, 4 * (size_t)m->P, m->L, 4 * (size_t)m->Pp, 4 * (size_t)m->P, B,
                              mem == BN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return check_status(m, s, "bn_mlp_forward");
}

extern "C" int bn_mlp_loss_grad(bn_mlp* m, const uint8_t* orders, const uint32_t* pairs, const float* alpha, int B,
                                float* loss, int mem, void* stream)
{
    set_error(BN_OK, "");
    if (!m || !orders || !pairs || !alpha || B < 1) return set_error(BN_EINVAL, "bn_mlp_loss_grad: bad arguments");
    if (B > m->cap) return set_error(BN_EINVAL, "bn_mlp_loss_grad: B=%d above batch capacity %d", B, m->cap);
    cudaStream_t s = (cudaStream_t)stream;
    const void *d_o = nullptr, *d_p = nullptr, *d_a = nullptr;
    int rc;
    if ((rc = stage_in(m->stage_orders, orders, (size_t)B * m->n, mem, s, &d_o)) ||
        (rc = stage_in(m->stage_pairs, pairs, 4 * (size_t)B, mem, s, &d_p)) ||
        (rc = stage_in(m->stage_alpha, alpha, 4 * (size_t)B, mem, s, &d_a)))
        return rc;
    if ((rc = mlp_loss_grad_dev(m, (const uint8_t*)d_o, (const uint32_t*)d_p, (const float*)d_a, B, s))) return rc;
    if (loss)
        BN_CUDA(cudaMemcpyAsync(loss, m->loss, 4, mem == BN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return check_status(m, s, "bn_mlp_loss_grad");
}

extern "C" int bn_mlp_adam_step(bn_mlp* m, void* stream)
{
    set_error(BN_OK, "");
    if (!m) return set_error(BN_EINVAL, "bn_mlp_adam_step: NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = mlp_adam_dev(m, s);
    if (rc) return rc;
    BN_CUDA(cudaStreamSynchronize(s));
    return BN_OK;
}

extern "C" int bn_mlp_read(const bn_mlp* m, int what, float* out, int mem, void* stream)
{
    set_error(BN_OK, "");
    if (!m || !out) return set_error(BN_EINVAL, "bn_mlp_read: NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const bool grad = what >= BN_MLP_GRAD_E;
    const int w = grad ? what - BN_MLP_GRAD_E : what;
    const float* src = nullptr;
    size_t rows = 1, cols = 0, spitch = 0;
    switch (w) {
        case BN_MLP_E: src = grad ? m->gE : m->E; rows = m->n; cols = m->d; spitch = m->d; break;
        case BN_MLP_W1: src = grad ? m->gW1 : m->W1; rows = m->H; cols = m->nd; spitch = m->ndp; break;
        case BN_MLP_B1: src = grad ? m->gb1 : m->b1; cols = m->H; spitch = cols; break;
        case BN_MLP_W2: src = grad ? m->gW2 : m->W2; rows = m->H; cols = m->H; spitch = m->H; break;
        case BN_MLP_B2: src = grad ? m->gb2 : m->b2; cols = m->H; spitch = cols; break;
        case BN_MLP_W3: src = grad ? m->gW3 : m->W3; rows = m->P; cols = m->H; spitch = m->H; break;
        case BN_MLP_B3: src = grad ? m->gb3 : m->b3; cols = m->P; spitch = cols; break;
        default: return set_error(BN_EINVAL, "bn_mlp_read: unknown tensor %d", what);
    }
    BN_CUDA(cudaMemcpy2DAsync(out, 4 * cols, src, 4 * spitch, 4 * cols, rows,
                              mem == BN_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    return BN_OK;
}

extern "C" void bn_mlp_free(bn_mlp* m)
{
    if (!m) return;
    cudaFree(m->block);
    delete m;
}

extern "C" int bn_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K, void* stream)
{
    set_error(BN_OK, "");
    if (!A || !B || !C) return set_error(BN_EINVAL, "bn_gemm_bf16: NULL");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* st = nullptr;
    BN_CUDA(cudaMallocAsync((void**)&st, 4, s));
    BN_CUDA(cudaMemsetAsync(st, 0, 4, s));
    int rc = gemm_tc((const bf16*)A, K, (const bf16*)B, K, C, N, M, N, K, st, s, nullptr, 0);
    uint32_t h = 0;
    if (!rc) {
        BN_CUDA(cudaMemcpyAsync(&h, st, 4, cudaMemcpyDeviceToHost, s));
    }
    cudaFreeAsync(st, s);
    BN_CUDA(cudaStreamSynchronize(s));
    if (rc) return rc;
    if (h & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_gemm_bf16: a bounded device wait expired");
    return BN_OK;
}
