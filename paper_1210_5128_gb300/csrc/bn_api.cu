// bn_api.cu -- error state, launch accounting, device properties, rank helpers.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "bn_internal.cuh"

namespace bn {

static thread_local char t_err[512] = "";
static std::atomic<int64_t> g_launches{0};

int set_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line)
{
    const char* base = strrchr(file, '/');
    set_error(e == cudaErrorMemoryAllocation ? BN_ENOMEM : BN_ECUDA, "%s failed: %s (%s:%d)", what,
              cudaGetErrorString(e), base ? base + 1 : file, line);
    return e == cudaErrorMemoryAllocation ? BN_ENOMEM : BN_ECUDA;
}

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int device_id()
{
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

unsigned long long context_id()
{
    typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
    typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

bool first_in_context(unsigned long long* slots)
{
    static std::mutex mu;
    const int d = device_id();
    if (d < 0 || d >= 64) return true;
    const unsigned long long id = context_id();
    std::lock_guard<std::mutex> g(mu);
    if (id != 0 && slots[d] == id) return false;
    slots[d] = id;
    return true;
}

int sm_count()
{
    static std::mutex mu;
    static int cache[64] = {0};
    int d = device_id();
    std::lock_guard<std::mutex> g(mu);
    if (d >= 0 && d < 64 && cache[d]) return cache[d];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    if (v <= 0) v = 1;
    if (d >= 0 && d < 64) cache[d] = v;
    return v;
}

// A wait that can only run out: an mbarrier nobody arrives at, and a global flag nobody
// sets, each waited on with the same bounded helpers the kernels use.
__global__ void k_selftest_wait(const volatile uint32_t* flag, uint64_t timeout_ns, uint32_t* status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait_bounded(&bar, 0, timeout_ns)) atomicOr(status, STATUS_TIMEOUT);
        const uint64_t t0 = global_timer_ns();
        while (*flag == 0u) {
            if (global_timer_ns() - t0 > timeout_ns) {
                atomicOr(status, STATUS_TIMEOUT << 1);
                break;
            }
        }
    }
}

}  // namespace bn

extern "C" {

int bn_selftest_timeout(int64_t timeout_ns, void* stream)
{
    bn::t_err[0] = 0;
    if (timeout_ns <= 0 || timeout_ns > 2000000000LL)
        return bn::set_error(BN_EINVAL, "bn_selftest_timeout: timeout must be in (0, 2 s]");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* d = nullptr;
    BN_CUDA(cudaMallocAsync((void**)&d, 8, s));
    BN_CUDA(cudaMemsetAsync(d, 0, 8, s));
    bn::k_selftest_wait<<<1, 32, 0, s>>>(d, (uint64_t)timeout_ns, d + 1);
    cudaError_t le = cudaGetLastError();
    uint32_t h = 0;
    if (le == cudaSuccess) {
        bn::count_launches(1);
        le = cudaMemcpyAsync(&h, d + 1, 4, cudaMemcpyDeviceToHost, s);
    }
    cudaFreeAsync(d, s);
    if (le != cudaSuccess) return bn::cuda_fail(le, "k_selftest_wait", __FILE__, __LINE__);
    BN_CUDA(cudaStreamSynchronize(s));
    if (h == (bn::STATUS_TIMEOUT | (bn::STATUS_TIMEOUT << 1)))
        return bn::set_error(BN_ETIMEOUT, "bn_selftest_timeout: both bounded waits gave up as intended");
    return bn::set_error(BN_ECUDA, "bn_selftest_timeout: unexpected status %u", h);
}

const char* bn_last_error(void) { return bn::t_err; }

const char* bn_version(void) { return "bngpu 0.1 (sm_103a)"; }

int64_t bn_kernel_launches(void) { return bn::g_launches.load(); }

int bn_unrank(int N, int k, int64_t rank, uint64_t* mask)
{
    bn::t_err[0] = 0;
    if (N < 0 || N > 63 || k < 0 || !mask) return bn::set_error(BN_EINVAL, "bn_unrank: bad arguments");
    if (k > N) k = N;
    int64_t S = bn::num_sets_host(N, k);
    if (rank < 0 || rank >= S) return bn::set_error(BN_EINVAL, "bn_unrank: rank %lld out of [0, %lld)",
                                                    (long long)rank, (long long)S);
    int j = 0;
    while (rank >= (int64_t)bn::h_binom.v[N][j]) { rank -= (int64_t)bn::h_binom.v[N][j]; ++j; }
    uint64_t m = 0;
    for (int t = j; t >= 1; --t) {
        int a = N - 1;
        while ((int64_t)bn::h_binom.v[a][t] > rank) --a;
        m |= 1ull << a;
        rank -= (int64_t)bn::h_binom.v[a][t];
    }
    *mask = m;
    return BN_OK;
}

int bn_rank(int N, int k, uint64_t mask, int64_t* rank)
{
    bn::t_err[0] = 0;
    if (N < 0 || N > 63 || k < 0 || !rank) return bn::set_error(BN_EINVAL, "bn_rank: bad arguments");
    if (N < 64 && (mask >> N) != 0) return bn::set_error(BN_EINVAL, "bn_rank: mask has bits >= N");
    int j = __builtin_popcountll(mask);
    if (j > k) return bn::set_error(BN_EINVAL, "bn_rank: set larger than k");
    int64_t r = 0;
    for (int t = 0; t < j; ++t) r += (int64_t)bn::h_binom.v[N][t];
    int t = 1;
    for (int c = 0; c < N; ++c)
        if (mask >> c & 1) r += (int64_t)bn::h_binom.v[c][t++];
    *rank = r;
    return BN_OK;
}

}  // extern "C"
