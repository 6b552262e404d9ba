// Throughput of mad.wide.u32 (32 x 32 -> 64-bit multiply-add into a 64-bit
// accumulator), the instruction of the recurrence's limb products, on the
// current GPU.  Standalone program, not part of the library:
//
//   nvcc -O3 -gencode arch=compute_103a,code=sm_103a -o mad_wide_probe mad_wide_probe.cu && ./mad_wide_probe
//
// Each line reports mad.wide.u32 per SM per clock (at 2070 MHz) for 12 warps
// per SM and 16 independent accumulators per thread:
//  fixed      both multiplicands fixed (the issue ceiling),
//  one update one multiplicand rewritten once per 16 mad.wide,
//  all update all 16 second multiplicands rewritten every 16 mad.wide,
//  loop       the recurrence's loop: per j one 64-bit entry of M (two 28-bit
//             limbs) and four columns of W (two limbs each) from shared
//             memory, 16 mad.wide.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ void madw(uint64_t &acc, uint32_t a, uint32_t b) {
    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

template <int MODE>
__global__ void __launch_bounds__(512) k_regs(int iters, unsigned long long *out) {
    uint64_t S[16];
    for (int t = 0; t < 16; t++) S[t] = t;
    uint32_t a = threadIdx.x | 1;
    uint32_t B[16];
    for (int t = 0; t < 16; t++) B[t] = threadIdx.x * (t + 11);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int t = 0; t < 16; t++) madw(S[t], a, B[t]);
        if (MODE == 1) a += 1;
        if (MODE == 2)
#pragma unroll
            for (int t = 0; t < 16; t++) B[t] += 1;
    }
    uint64_t tot = a;
    for (int t = 0; t < 16; t++) tot += S[t] + B[t];
    if (tot == 42) out[0] = tot;
}

__global__ void __launch_bounds__(512) k_loop(int s, int nrows, int cs, int reps, unsigned long long *out) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint64_t *Ms = (uint64_t *)sm;
    uint2 *W = (uint2 *)(sm + ((nrows * s * 8 + 127) & ~127));
    for (int e = threadIdx.x; e < nrows * s; e += blockDim.x) Ms[e] = (0x9E3779B97F4A7C15ull * (e + 1)) >> 8;
    for (int e = threadIdx.x; e < s * cs; e += blockDim.x) W[e] = make_uint2(e * 2654435761u & 0xfffffff, e * 40503u & 0xfffffff);
    __syncthreads();
    const int items = nrows * (cs / 4);
    uint64_t tot = 0;
    for (int r = 0; r < reps; r++) {
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int rl = it % nrows, c0 = (it / nrows) * 4;
            uint64_t S[4][4] = {};
            const uint64_t *mp = Ms + rl;
            const uint4 *wp = (const uint4 *)(W + c0);
#pragma unroll 2
            for (int j = 0; j < s; j++) {
                const uint64_t m = *mp;
                mp += nrows;
                const uint32_t m0 = (uint32_t)m & 0xfffffff, m1 = (uint32_t)(m >> 28);
                const uint4 wa = wp[0], wb = wp[1];
                wp += cs / 2;
                madw(S[0][0], m0, wa.x); madw(S[0][1], m0, wa.y); madw(S[1][0], m0, wa.z); madw(S[1][1], m0, wa.w);
                madw(S[2][0], m0, wb.x); madw(S[2][1], m0, wb.y); madw(S[3][0], m0, wb.z); madw(S[3][1], m0, wb.w);
                madw(S[0][2], m1, wa.x); madw(S[0][3], m1, wa.y); madw(S[1][2], m1, wa.z); madw(S[1][3], m1, wa.w);
                madw(S[2][2], m1, wb.x); madw(S[2][3], m1, wb.y); madw(S[3][2], m1, wb.z); madw(S[3][3], m1, wb.w);
            }
            for (int a = 0; a < 4; a++)
                for (int t = 0; t < 4; t++) tot += S[a][t];
        }
        __syncthreads();
    }
    if (tot == 42) out[0] = tot;
}

static double rate(double ops, float ms, int sms) { return ops / (ms / 1e3) / sms / 2.07e9; }

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    unsigned long long *out;
    cudaMalloc(&out, 8);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 384, iters = 4096;
    void (*regs[3])(int, unsigned long long *) = {k_regs<0>, k_regs<1>, k_regs<2>};
    const char *names[3] = {"fixed", "one update", "all update"};
    for (int m = 0; m < 3; m++) {
        regs[m]<<<sms, threads>>>(16, out);
        cudaEventRecord(e0);
        regs[m]<<<sms, threads>>>(iters, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        printf("%-11s %6.1f mad.wide/clk/SM  %s\n", names[m], rate((double)sms * threads * iters * 16, ms, sms),
               cudaGetErrorString(cudaGetLastError()));
    }
    const int s = 220, nrows = 55, cs = 24, reps = 200;
    const size_t smem = ((nrows * s * 8 + 127) & ~127) + (size_t)s * cs * 8;
    cudaFuncSetAttribute(k_loop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_loop<<<sms, threads, smem>>>(s, nrows, cs, 1, out);
    cudaEventRecord(e0);
    k_loop<<<sms, threads, smem>>>(s, nrows, cs, reps, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    printf("%-11s %6.1f mad.wide/clk/SM  %s\n", "loop", rate((double)sms * reps * nrows * (cs / 4) * s * 16, ms, sms),
           cudaGetErrorString(cudaGetLastError()));
    return 0;
}
