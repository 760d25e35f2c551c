// probes.cu -- micro-benchmarks of the unit rates the BLS roofline is built from.
//
//   bls_probes [seconds_per_probe]
//
// Prints one JSON object per probe: rate per SM per clock, with the SM clock measured
// in-kernel (clock64 against globaltimer).  Probes:
//   fp32_fma     independent FP32 FMAs (8 chains per thread)
//   fp32x2_fma   packed fma.rn.f32x2 (4 chains, 2 lanes each)
//   fp64_fma     independent FP64 FMAs
//   smem_rmw     private-column histogram update: load 8 B, two adds, store 8 B per point
//   smem_rmw2    the same, two points per step with store forwarding
//   smem_red     private-column update with two shared-memory float atomic adds
//   smem_ired32  private-column update with two shared-memory 32-bit integer reductions
//   smem_ired64  private-column update with one shared-memory 64-bit integer reduction
//   smem_ired32p two 32-bit integer reductions per point into separate W and X planes
//                (4-byte entries, stride = threads: the 32 lanes of a warp hit 32 banks)
//   lds64        private-column 8-byte loads only
//   mufu_rcp     approximate reciprocals (8 chains per thread)
//   lds*/sts*_bw shared-memory bytes per SM per clock for 4, 8 and 16 bytes per lane
// The histogram probes run one block per SM (like the search kernel, whose shared
// histograms fill the SM) with 64, 128 or 192 threads.
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>
#include <stdint.h>

#define CK(x)                                                                     \
    do {                                                                          \
        cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) {                                                  \
            fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));              \
            exit(1);                                                              \
        }                                                                         \
    } while (0)

struct Stamp {
    long long c0, c1;
    unsigned long long t0, t1;
};

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void fp32_fma(int iters, float* out, Stamp* st)
{
    long long c0 = clock64();
    unsigned long long t0 = gtimer();
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = threadIdx.x * 1e-3f + q;
    const float m = 0.999f, c = 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __fmaf_rn(a[q], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) st[blockIdx.x] = Stamp{c0, clock64(), t0, gtimer()};
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__global__ void fp32x2_fma(int iters, float* out, Stamp* st)
{
    long long c0 = clock64();
    unsigned long long t0 = gtimer();
    unsigned long long a[4];
    float2 init;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        init = make_float2(threadIdx.x * 1e-3f + q, q + 0.5f);
        a[q] = *reinterpret_cast<unsigned long long*>(&init);
    }
    float2 mm = make_float2(0.999f, 0.999f), cc = make_float2(1e-4f, 1e-4f);
    const unsigned long long m = *reinterpret_cast<unsigned long long*>(&mm);
    const unsigned long long c = *reinterpret_cast<unsigned long long*>(&cc);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = fma2(a[q], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 v = *reinterpret_cast<float2*>(&a[q]);
        s += v.x + v.y;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) st[blockIdx.x] = Stamp{c0, clock64(), t0, gtimer()};
}

__global__ void fp64_fma(int iters, float* out, Stamp* st)
{
    long long c0 = clock64();
    unsigned long long t0 = gtimer();
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = threadIdx.x * 1e-3 + q;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __fma_rn(a[q], 0.999, 1e-4);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    if (threadIdx.x == 0) st[blockIdx.x] = Stamp{c0, clock64(), t0, gtimer()};
}

__global__ void mufu_rcp(int iters, float* out, Stamp* st)
{
    long long c0 = clock64();
    unsigned long long t0 = gtimer();
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = 1.0f + threadIdx.x * 1e-3f + q;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float r;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[q]));
            a[q] = __fadd_rn(r, 1.0f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) st[blockIdx.x] = Stamp{c0, clock64(), t0, gtimer()};
}

// Shared-memory bandwidth: every lane reads (or writes) W bytes per access at conflict-free
// consecutive addresses, 8 independent accesses per iteration.
template <int W, int STORE>
__global__ void smem_bw(int iters, float* out, Stamp* st)
{
    extern __shared__ __align__(16) float4 S4[];
    const int T = blockDim.x, t = threadIdx.x;
    const int span = 8 * T;   // elements of W bytes
    for (int i = t; i < span; i += T) S4[i] = make_float4(1.f, 2.f, 3.f, 4.f);
    __syncthreads();
    long long c0 = clock64();
    unsigned long long t0 = gtimer();
    float acc = 0.f;
    const unsigned base = (unsigned)__cvta_generic_to_shared(S4);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const unsigned a = base + (unsigned)((q * T + t) * W);
            if (STORE) {
                if (W == 4) asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(acc));
                if (W == 8) asm volatile("st.shared.v2.f32 [%0], {%1, %1};" ::"r"(a), "f"(acc));
                if (W == 16) asm volatile("st.shared.v4.f32 [%0], {%1, %1, %1, %1};" ::"r"(a), "f"(acc));
            } else {
                float x, y, z, w;
                if (W == 4) { asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x) : "r"(a)); acc += x; }
                if (W == 8) { asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a)); acc += x; }
                if (W == 16) { asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a)); acc += x; }
            }
        }
        acc *= 0.5f;
    }
    long long c1 = clock64();
    unsigned long long t1 = gtimer();
    out[blockIdx.x * blockDim.x + t] = acc;
    if (t == 0) st[blockIdx.x] = Stamp{c0, c1, t0, t1};
}

// Private-column histogram of 128 bins (float2 entries, stride = blockDim.x).
template <int MODE>
__global__ void smem_hist(int iters, float* out, Stamp* st)
{
    extern __shared__ float2 H[];
    const int T = blockDim.x, t = threadIdx.x;
    for (int b = 0; b < 128; ++b) H[b * T + t] = make_float2(0.f, 0.f);
    __syncthreads();
    long long c0 = clock64();
    unsigned long long t0 = gtimer();
    uint32_t x = 12345u + 977u * t + 131u * blockIdx.x;
    float acc = 0.f;
    const float w = 1e-3f, wx = -2e-5f;
    if (MODE == 0) {            // rmw, one point at a time
        for (int i = 0; i < iters; ++i) {
            x = x * 1664525u + 1013904223u;
            float2* p = &H[(x >> 25) * T + t];
            float2 v = *p;
            v.x += w; v.y += wx;
            *p = v;
        }
    } else if (MODE == 1) {     // rmw, two points per step with store forwarding
        for (int i = 0; i < iters; i += 2) {
            x = x * 1664525u + 1013904223u;
            const uint32_t b0 = x >> 25;
            x = x * 1664525u + 1013904223u;
            const uint32_t b1 = x >> 25;
            float2* p0 = &H[b0 * T + t];
            float2* p1 = &H[b1 * T + t];
            float2 h0 = *p0, h1 = *p1, v0, v1;
            v0.x = h0.x + w; v0.y = h0.y + wx;
            const bool same = b0 == b1;
            v1.x = (same ? v0.x : h1.x) + w;
            v1.y = (same ? v0.y : h1.y) + wx;
            *p0 = v0;
            *p1 = v1;
        }
    } else if (MODE == 2) {     // two shared-memory float atomic adds per point
        float* Hf = reinterpret_cast<float*>(H);
        for (int i = 0; i < iters; ++i) {
            x = x * 1664525u + 1013904223u;
            const uint32_t e = ((x >> 25) * T + t) * 2;
            atomicAdd(&Hf[e], w);
            atomicAdd(&Hf[e + 1], wx);
        }
    } else if (MODE == 4) {     // two 32-bit integer reductions per point (fixed point)
        const unsigned base = (unsigned)__cvta_generic_to_shared(H);
        for (int i = 0; i < iters; ++i) {
            x = x * 1664525u + 1013904223u;
            const unsigned a = base + ((x >> 25) * T + t) * 8u;
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(x & 0xffffu) : "memory");
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a + 4u), "r"(x >> 20) : "memory");
        }
    } else if (MODE == 5) {     // one 64-bit integer reduction per point (packed fields)
        const unsigned base = (unsigned)__cvta_generic_to_shared(H);
        for (int i = 0; i < iters; ++i) {
            x = x * 1664525u + 1013904223u;
            const unsigned a = base + ((x >> 25) * T + t) * 8u;
            const unsigned long long v = ((unsigned long long)(x >> 20) << 32) | (x & 0xffffu);
            asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
        }
    } else if (MODE == 6) {     // two 32-bit reductions per point, W and X planes
        const unsigned base = (unsigned)__cvta_generic_to_shared(H);
        const unsigned plane = 128u * T * 4u;
        for (int i = 0; i < iters; ++i) {
            x = x * 1664525u + 1013904223u;
            const unsigned a = base + ((x >> 25) * T + t) * 4u;
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(x & 0xffffu) : "memory");
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a + plane), "r"(x >> 20) : "memory");
        }
    } else {                    // loads only
        for (int i = 0; i < iters; ++i) {
            x = x * 1664525u + 1013904223u;
            float2 v = H[(x >> 25) * T + t];
            acc += v.x + v.y;
        }
    }
    long long c1 = clock64();
    unsigned long long t1 = gtimer();
    __syncthreads();
    float2 v = H[(x >> 25) * T + t];
    out[blockIdx.x * blockDim.x + t] = v.x + v.y + acc;
    if (t == 0) st[blockIdx.x] = Stamp{c0, c1, t0, t1};
}

struct Result {
    double ms, clk_mhz, per_sm_clk;
};

template <class F>
static Result run(F launch, int blocks, double ops, Stamp* d_st, int sms)
{
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    launch();  // warm-up
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(a));
    launch();
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    Stamp* h = new Stamp[blocks];
    CK(cudaMemcpy(h, d_st, sizeof(Stamp) * blocks, cudaMemcpyDeviceToHost));
    double cyc = 0, ns = 0;
    for (int i = 0; i < blocks; ++i) {
        cyc += (double)(h[i].c1 - h[i].c0);
        ns += (double)(h[i].t1 - h[i].t0);
    }
    delete[] h;
    Result r;
    r.ms = ms;
    r.clk_mhz = cyc / ns * 1e3;
    // ops per SM per clock over the kernel time
    r.per_sm_clk = ops / (sms * (ms * 1e-3) * r.clk_mhz * 1e6);
    return r;
}

int main(int argc, char** argv)
{
    double scale = argc > 1 ? atof(argv[1]) : 1.0;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* out;
    Stamp* st;
    const int maxblocks = sms * 16;
    CK(cudaMalloc(&out, sizeof(float) * maxblocks * 1024));
    CK(cudaMalloc(&st, sizeof(Stamp) * maxblocks));

    {   // FP32 FMA: 8 blocks x 256 threads per SM
        const int blocks = sms * 8, T = 256, it = (int)(20000 * scale);
        Result r = run([&] { fp32_fma<<<blocks, T>>>(it, out, st); }, blocks, (double)blocks * T * it * 8, st, sms);
        printf("{\"probe\": \"fp32_fma\", \"ms\": %.3f, \"clk_mhz\": %.0f, \"fma_per_sm_clk\": %.2f}\n", r.ms, r.clk_mhz, r.per_sm_clk);
    }
    {
        const int blocks = sms * 8, T = 256, it = (int)(20000 * scale);
        Result r = run([&] { fp32x2_fma<<<blocks, T>>>(it, out, st); }, blocks, (double)blocks * T * it * 8, st, sms);
        printf("{\"probe\": \"fp32x2_fma\", \"ms\": %.3f, \"clk_mhz\": %.0f, \"fma_per_sm_clk\": %.2f}\n", r.ms, r.clk_mhz, r.per_sm_clk);
    }
    {
        const int blocks = sms * 8, T = 256, it = (int)(1000 * scale);
        Result r = run([&] { fp64_fma<<<blocks, T>>>(it, out, st); }, blocks, (double)blocks * T * it * 8, st, sms);
        printf("{\"probe\": \"fp64_fma\", \"ms\": %.3f, \"clk_mhz\": %.0f, \"fma_per_sm_clk\": %.2f}\n", r.ms, r.clk_mhz, r.per_sm_clk);
    }
    {
        const int blocks = sms * 8, T = 256, it = (int)(4000 * scale);
        Result r = run([&] { mufu_rcp<<<blocks, T>>>(it, out, st); }, blocks, (double)blocks * T * it * 8, st, sms);
        printf("{\"probe\": \"mufu_rcp\", \"ms\": %.3f, \"clk_mhz\": %.0f, \"rcp_per_sm_clk\": %.2f}\n", r.ms, r.clk_mhz, r.per_sm_clk);
    }
    {   // shared-memory bandwidth, 8 warps per SM (two 128-thread blocks)
        const int T = 128, blocks = sms * 2, it = (int)(20000 * scale);
        const size_t smem = (size_t)8 * T * 16;
        auto runbw = [&](const char* nm, int W, auto k) {
            CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            Result r = run([&] { k<<<blocks, T, smem>>>(it, out, st); }, blocks,
                           (double)blocks * T * it * 8 * W, st, sms);
            printf("{\"probe\": \"%s\", \"ms\": %.3f, \"clk_mhz\": %.0f, \"bytes_per_sm_clk\": %.1f}\n", nm, r.ms,
                   r.clk_mhz, r.per_sm_clk);
        };
        runbw("lds32_bw", 4, smem_bw<4, 0>);
        runbw("lds64_bw", 8, smem_bw<8, 0>);
        runbw("lds128_bw", 16, smem_bw<16, 0>);
        runbw("sts32_bw", 4, smem_bw<4, 1>);
        runbw("sts64_bw", 8, smem_bw<8, 1>);
        runbw("sts128_bw", 16, smem_bw<16, 1>);
    }
    const char* names[7] = {"smem_rmw", "smem_rmw2", "smem_red", "lds64", "smem_ired32",
                            "smem_ired64", "smem_ired32p"};
    const int Ts[3] = {64, 128, 192};
    for (int mode = 0; mode < 7; ++mode) {
        for (int ti = 0; ti < 3; ++ti) {
            const int T = Ts[ti];
            const size_t smem = (size_t)128 * T * sizeof(float2);
            const int blocks = sms, it = (int)(40000 * scale);
            auto k = mode == 0 ? smem_hist<0> : mode == 1 ? smem_hist<1> : mode == 2 ? smem_hist<2>
                   : mode == 3 ? smem_hist<3> : mode == 4 ? smem_hist<4> : mode == 5 ? smem_hist<5>
                   : smem_hist<6>;
            CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            Result r = run([&] { k<<<blocks, T, smem>>>(it, out, st); }, blocks, (double)blocks * T * it, st, sms);
            printf("{\"probe\": \"%s\", \"threads_per_sm\": %d, \"ms\": %.3f, \"clk_mhz\": %.0f, \"points_per_sm_clk\": %.3f}\n",
                   names[mode], T, r.ms, r.clk_mhz, r.per_sm_clk);
        }
    }
    CK(cudaFree(out));
    CK(cudaFree(st));
    return 0;
}
