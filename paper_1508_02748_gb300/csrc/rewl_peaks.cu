// Microbenchmarks of the rates that bound the sampling kernels on the GPU
// they run on: issue of independent integer logic (lop3), integer add,
// integer multiply-add and float fma instructions, the latency of a chain of
// dependent integer adds, and the read bandwidth of shared memory and of the
// L2 cache.  Each kernel is timed with CUDA events on the caller's stream;
// every result is per second of device time (the SM clock is whatever the
// GPU runs at meanwhile; the caller samples it).
#include <cstring>

#include "rewl_internal.cuh"

namespace rewl {

namespace {

constexpr int CHAINS = 8;          // independent dependency chains per thread
constexpr int UNROLL = 16;

// op: 0 lop3.b32, 1 add.u32, 2 mad.lo.u32, 3 fma.rn.f32
template <int OP>
__global__ void __launch_bounds__(256) k_issue(uint32_t *sink, int iters, uint32_t seed)
{
    uint32_t r[CHAINS];
    float f[CHAINS];
    #pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
        r[c] = seed ^ (threadIdx.x * 0x9E3779B9u + c);
        f[c] = (float)(r[c] & 1023u) * 0.001f;
    }
    const uint32_t k1 = seed | 1u, k2 = seed >> 3;
    const float g1 = 0.999f, g2 = 0.001f;
    for (int i = 0; i < iters; ++i) {
        #pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            #pragma unroll
            for (int c = 0; c < CHAINS; ++c) {
                if (OP == 0) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(r[c]) : "r"(k1), "r"(k2));
                if (OP == 1) asm volatile("add.u32 %0, %0, %1;" : "+r"(r[c]) : "r"(k1));
                if (OP == 2) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(r[c]) : "r"(k1), "r"(k2));
                if (OP == 3) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[c]) : "f"(g1), "f"(g2));
            }
        }
    }
    uint32_t x = 0;
    #pragma unroll
    for (int c = 0; c < CHAINS; ++c) x ^= r[c] ^ __float_as_uint(f[c]);
    if (x == seed) sink[0] = x;     // keeps the chains live
}

// One dependent chain of adds per thread, one warp per SM sub-partition.
__global__ void k_dep_add(uint32_t *sink, int iters, uint32_t seed, unsigned long long *cycles)
{
    uint32_t r = seed ^ threadIdx.x;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        #pragma unroll
        for (int u = 0; u < UNROLL; ++u) asm volatile("add.u32 %0, %0, %1;" : "+r"(r) : "r"(seed));
    }
    const long long t1 = clock64();
    if (r == seed) sink[0] = r;
    if (blockIdx.x == 0 && threadIdx.x == 0) *cycles = (unsigned long long)(t1 - t0);
}

// Shared-memory reads: 16-byte vector loads, consecutive lanes on
// consecutive 16-byte words (no bank conflicts), 48 KiB per block.
__global__ void __launch_bounds__(512) k_smem(uint32_t *sink, int iters)
{
    __shared__ uint4 buf[3072];
    for (int k = threadIdx.x; k < 3072; k += blockDim.x) buf[k] = make_uint4(k, k * 3, k * 5, k * 7);
    __syncthreads();
    uint32_t x = 0;
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        #pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const uint4 v = buf[idx];
            x ^= v.x ^ v.y ^ v.z ^ v.w;
            idx += 512;
            if (idx >= 3072) idx -= 3072;
        }
    }
    if (x == 0x12345678u) sink[0] = x;
}

// L2 reads: 16-byte loads that bypass L1 (ld.global.cg) over a buffer that
// fits in L2, grid-stride, several passes.
__global__ void __launch_bounds__(256) k_l2(const uint4 *buf, size_t n, int passes, uint32_t *sink)
{
    uint32_t x = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
            uint4 v;
            asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(buf + i));
            x ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (x == 0x12345678u) sink[0] = x;
}

__global__ void k_fill(uint4 *buf, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        buf[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 7), 3u, 5u);
}

}  // namespace

}  // namespace rewl

using namespace rewl;

namespace {

// Milliseconds of one launch of `launch` on s (after one untimed launch).
template <class F>
int time_ms(cudaStream_t s, F launch, float *ms)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return REWL_E_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return REWL_E_CUDA; }
    launch();
    cudaEventRecord(a, s);
    launch();
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e == cudaSuccess ? REWL_OK : REWL_E_CUDA;
}

}  // namespace

extern "C" int rewl_measure_peaks(void *d_scratch, size_t scratch_bytes, void *stream, rewl_peaks *out)
{
    if (!out || !d_scratch || scratch_bytes < ((size_t)64 << 20) + 4096 || ((uintptr_t)d_scratch & 255u))
        return REWL_E_INVALID;
    std::memset(out, 0, sizeof(*out));
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return REWL_E_CUDA;
    uint32_t *sink = (uint32_t *)d_scratch;
    unsigned long long *cyc = (unsigned long long *)((char *)d_scratch + 256);
    uint4 *buf = (uint4 *)((char *)d_scratch + 4096);
    const size_t nbuf = ((size_t)64 << 20) / sizeof(uint4);
    float ms = 0;
    int rc;

    // issue rates: 8 warps per block, 4 blocks per SM, CHAINS x UNROLL x iters ops per thread
    const int blocks = sms * 4, threads = 256, iters = 2048;
    const double ops = (double)blocks * threads * CHAINS * UNROLL * iters;
    double *dst[4] = {&out->lop3_ops_per_s, &out->iadd_ops_per_s, &out->imad_ops_per_s, &out->ffma_ops_per_s};
    for (int op = 0; op < 4; ++op) {
        rc = time_ms(s, [&] {
            if (op == 0) k_issue<0><<<blocks, threads, 0, s>>>(sink, iters, 0x2545F491u);
            if (op == 1) k_issue<1><<<blocks, threads, 0, s>>>(sink, iters, 0x2545F491u);
            if (op == 2) k_issue<2><<<blocks, threads, 0, s>>>(sink, iters, 0x2545F491u);
            if (op == 3) k_issue<3><<<blocks, threads, 0, s>>>(sink, iters, 0x2545F491u);
        }, &ms);
        if (rc) return rc;
        *dst[op] = ops / (ms * 1e-3);
    }

    // dependent adds: cycles per add of one chain
    {
        const int it = 4096;
        rc = time_ms(s, [&] { k_dep_add<<<sms, 128, 0, s>>>(sink, it, 7u, cyc); }, &ms);
        if (rc) return rc;
        unsigned long long c = 0;
        if (cudaMemcpyAsync(&c, cyc, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return REWL_E_CUDA;
        out->dep_iadd_cycles = (double)c / ((double)it * UNROLL);
    }

    // shared memory: 512 threads x 16 B x UNROLL x iters per block, 4 blocks per SM
    {
        const int it = 4096, b = sms * 4;
        rc = time_ms(s, [&] { k_smem<<<b, 512, 0, s>>>(sink, it); }, &ms);
        if (rc) return rc;
        out->smem_bytes_per_s = (double)b * 512 * 16 * UNROLL * it / (ms * 1e-3);
    }

    // L2: 64 MiB read 8 times with L1 bypassed (the first, untimed launch warms L2)
    {
        k_fill<<<sms * 8, 256, 0, s>>>(buf, nbuf);
        const int passes = 8;
        rc = time_ms(s, [&] { k_l2<<<sms * 8, 256, 0, s>>>(buf, nbuf, passes, sink); }, &ms);
        if (rc) return rc;
        out->l2_bytes_per_s = (double)nbuf * sizeof(uint4) * passes / (ms * 1e-3);
    }
    out->sms = sms;
    return REWL_OK;
}
