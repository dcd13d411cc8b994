// bn_internal.cuh -- device helpers and shared host declarations of the CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bn.h"

namespace bn {

constexpr int MAXN = 64;            // nodes per network (candidate masks are 64-bit)
constexpr int MAXK = 12;            // parents per set the table builder supports
constexpr int MAX_CELLS = 4096;     // q * r cells of one count table
constexpr int SUBQ = 256;           // per-node table stride is a multiple of this

// ---------------------------------------------------------------------------------
// Host-side error state, launch accounting, per-device properties (bn_api.cu)
// ---------------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
void count_launches(int64_t k);
int sm_count();                      // SMs of the current device
int device_id();
// Identity of the calling thread's current CUDA context (0 when the driver cannot say).
unsigned long long context_id();
// True the first time it is called in the current context of the current device with
// this call site's `slots` (64 zero-initialised entries): per-context set-up, such as a
// kernel's shared-memory attribute, which a context destroyed and created again loses.
bool first_in_context(unsigned long long* slots);

#define BN_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess) return ::bn::cuda_fail(_e, #call, __FILE__, __LINE__);  \
    } while (0)

#define BN_LAUNCH_CHECK(what)                                                          \
    do {                                                                               \
        cudaError_t _e = cudaGetLastError();                                           \
        if (_e != cudaSuccess) return ::bn::cuda_fail(_e, what, __FILE__, __LINE__);   \
        ::bn::count_launches(1);                                                       \
    } while (0)

inline int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

// ---------------------------------------------------------------------------------
// Binomial coefficients C(a, t), 0 <= a, t <= 64, built at compile time.
// ---------------------------------------------------------------------------------
struct BinomTable {
    uint64_t v[65][65];
};
constexpr BinomTable make_binom()
{
    BinomTable b{};
    for (int a = 0; a <= 64; ++a) {
        b.v[a][0] = 1;
        for (int t = 1; t <= 64; ++t)
            b.v[a][t] = (a == 0) ? 0 : b.v[a - 1][t - 1] + b.v[a - 1][t];
    }
    return b;
}
static __constant__ BinomTable c_binom = make_binom();
constexpr BinomTable h_binom = make_binom();

// sets of size <= k drawn from N candidates
inline int64_t num_sets_host(int N, int k)
{
    int64_t s = 0;
    for (int j = 0; j <= k && j <= N; ++j) s += (int64_t)h_binom.v[N][j];
    return s;
}

// ---------------------------------------------------------------------------------
// Order-preserving int64 key of an FP64 score (an involution on the bit pattern):
// for finite doubles x < y  <=>  key(x) < key(y) as signed integers.
// ---------------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t key_from_bits(uint64_t b)
{
    int64_t x = (int64_t)b;
    return x ^ ((x >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__host__ __device__ __forceinline__ uint64_t bits_from_key(int64_t k)
{
    return (uint64_t)(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}
constexpr int64_t KEY_NONE = (int64_t)0x8000000000000000ULL;   // below every finite key

__device__ __forceinline__ double key_to_double(int64_t k)
{
    return __longlong_as_double((long long)bits_from_key(k));
}
__device__ __forceinline__ int64_t double_to_key(double d)
{
    return key_from_bits((uint64_t)__double_as_longlong(d));
}

// ---------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------------
struct U64x4 {
    uint64_t x[4];
};
__device__ __forceinline__ U64x4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                            uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    U64x4 o;
    o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
    return o;
}

// pair index p in [0, n(n-1)/2) -> positions a < b, lexicographic pair order.  Row a
// starts at st(a) = a (2n - a - 1) / 2; a = max{a : st(a) <= p} from the quadratic's
// root in FP32, then made exact with integer comparisons.
__device__ __forceinline__ void pair_decode(int n, uint64_t p, int& a, int& b)
{
    const int ip = (int)p;
    const float m = (float)(2 * n - 1);
    int x = (int)floorf(0.5f * (m - sqrtf(fmaxf(m * m - 8.0f * (float)ip, 0.0f))));
    x = max(0, min(x, n - 2));
    while (x > 0 && x * (2 * n - x - 1) / 2 > ip) --x;
    while (x + 1 <= n - 2 && (x + 1) * (2 * n - x - 2) / 2 <= ip) ++x;
    a = x;
    b = x + 1 + (ip - x * (2 * n - x - 1) / 2);
}

// ---------------------------------------------------------------------------------
// 128-bit fixed point with 64 fractional bits (exact sums of FP64 lgamma terms)
// ---------------------------------------------------------------------------------
typedef unsigned __int128 fx128;

__device__ __forceinline__ fx128 fx_from_double(double v)
{
    bool neg = v < 0.0;
    double a = fabs(v);
    double ip = floor(a);
    double fr = a - ip;                                   // exact
    uint64_t lo = __double2ull_rz(fr * 18446744073709551616.0);   // * 2^64, exact scaling
    uint64_t hi = (uint64_t)ip;
    fx128 u = ((fx128)hi << 64) | (fx128)lo;
    return neg ? (fx128)0 - u : u;
}
__device__ __forceinline__ double fx_to_double(fx128 u)
{
    int64_t hi = (int64_t)(uint64_t)(u >> 64);
    uint64_t lo = (uint64_t)u;
    return __dadd_rn((double)hi, __dmul_rn(__ull2double_rn(lo), 5.421010862427522170037e-20));
}

// ---------------------------------------------------------------------------------
// Bounded waits, mbarriers and 1-D bulk (TMA) copies
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// one plain arrival (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// wait for the phase with the given parity; false after ~timeout_ns (the caller reports)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > timeout_ns) return false;
    }
    return true;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// global -> this CTA's shared memory, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Device-side status word written by kernels that give up a bounded wait.
constexpr uint32_t STATUS_TIMEOUT = 1u;
constexpr uint32_t STATUS_BADINPUT = 2u;
constexpr uint64_t WAIT_TIMEOUT_NS = 1000000000ull;   // 1 s

}  // namespace bn
