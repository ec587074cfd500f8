// Measured ALU rates of this GPU, for the roofline of the FP32-bound field
// kernels (not part of the method): dependent chains of packed f32x2 FMAs,
// of rsqrt.approx, and the all-pairs kernels' mixes (twelve FP32 lane-operations
// per rsqrt one-sided; sixteen per rsqrt symmetric, fourteen when the tiles'
// charges factor out), on every SM at once.  Rates per SM per clock come from the
// blocks' own clock64 spans; the TFLOP/s figure from CUDA events.
#include "obem_internal.cuh"
#include "field_common.cuh"

#define PK_THREADS 256
#define PK_BLOCKS_PER_SM 4      // 4 x 256 threads x <= 64 registers: one wave
#define PK_CHAINS 8

template <int MODE>   // 0: packed FMA chains, 1: rsqrt chains, 2 / 3 / 4: 6 / 8 / 7 packed FMAs (12 / 16 / 14 lane-ops) per rsqrt
__global__ void __launch_bounds__(PK_THREADS, PK_BLOCKS_PER_SM) alu_rate_kernel(int iters, float *sink,
                                                                               long long *cycles)
{
    const float s0 = 1.0f + 1e-3f * threadIdx.x;
    u64 P[PK_CHAINS];
    float S[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) { P[i] = pk(s0 + i, s0 - i); S[i] = s0 + 0.5f * i; }
    const u64 m = pk(0.999f, 0.998f), a = pk(1e-3f, 2e-3f);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int i = 0; i < PK_CHAINS; ++i) {
                if (MODE == 0) P[i] = fma2(P[i], m, a);
                if (MODE == 1) S[i] = rsq(S[i]);
                if (MODE >= 2) {
                    P[i] = fma2(P[i], m, a); P[i] = fma2(P[i], m, a); P[i] = fma2(P[i], m, a);
                    P[i] = fma2(P[i], m, a); P[i] = fma2(P[i], m, a); P[i] = fma2(P[i], m, a);
                    if (MODE >= 3) P[i] = fma2(P[i], m, a);
                    if (MODE == 3) P[i] = fma2(P[i], m, a);
                    S[i] = rsq(S[i]);
                }
            }
        }
    }
    const long long t1 = clock64();
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) {
        float x, y;
        upk(P[i], x, y);
        acc += x + y + S[i];
    }
    sink[blockIdx.x * PK_THREADS + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int MODE>
static int alu_rate(obem_ctx *c, int sms, float *sink, long long *cyc, long long *hcyc, cudaStream_t s,
                    double &per_sm_clk, double &per_s)
{
    const int blocks = sms * PK_BLOCKS_PER_SM, iters = MODE == 0 ? 8192 : 2048;
    alu_rate_kernel<MODE><<<blocks, PK_THREADS, 0, s>>>(64, sink, cyc);   // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    alu_rate_kernel<MODE><<<blocks, PK_THREADS, 0, s>>>(iters, sink, cyc);
    cudaEventRecord(e1, s);
    OBEM_LAUNCH(c);
    OBEM_CUDA(c, cudaMemcpyAsync(hcyc, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost, s));
    OBEM_CUDA(c, cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    long long mx = 1;
    for (int b = 0; b < blocks; ++b) mx = hcyc[b] > mx ? hcyc[b] : mx;
    // operations per thread: FP32 lane-ops for modes 0 and 2, rsqrt for mode 1
    const double ops = (double)iters * 8 * PK_CHAINS * (MODE == 0 ? 2 : MODE == 1 ? 1 : MODE == 2 ? 12 : MODE == 3 ? 16 : 14);
    const double total = ops * (double)blocks * PK_THREADS;
    per_sm_clk = total / sms / (double)mx;
    per_s = total / (ms * 1e-3);
    return OBEM_OK;
}

extern "C" int obem_alu_rates(obem_ctx *c, double *out, obem_stream stream)
{
    if (!c || !out) return OBEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    OBEM_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int blocks = sms * PK_BLOCKS_PER_SM;
    float *sink = NULL;
    long long *cyc = NULL;
    OBEM_CUDA(c, cudaMalloc((void **)&sink, sizeof(float) * (size_t)blocks * PK_THREADS));
    if (cudaMalloc((void **)&cyc, sizeof(long long) * blocks) != cudaSuccess) {
        cudaFree(sink);
        return obem_fail(c, OBEM_ERR_CUDA, "alu rates: allocation failed");
    }
    long long *hcyc = (long long *)malloc(sizeof(long long) * blocks);
    double r0 = 0, f0 = 0, r1 = 0, f1 = 0, r2 = 0, f2 = 0, r3 = 0, f3 = 0, r4 = 0, f4 = 0;
    int rc = hcyc ? OBEM_OK : OBEM_ERR_ARG;
    if (rc == OBEM_OK) rc = alu_rate<0>(c, sms, sink, cyc, hcyc, s, r0, f0);
    if (rc == OBEM_OK) rc = alu_rate<1>(c, sms, sink, cyc, hcyc, s, r1, f1);
    if (rc == OBEM_OK) rc = alu_rate<2>(c, sms, sink, cyc, hcyc, s, r2, f2);
    if (rc == OBEM_OK) rc = alu_rate<3>(c, sms, sink, cyc, hcyc, s, r3, f3);
    if (rc == OBEM_OK) rc = alu_rate<4>(c, sms, sink, cyc, hcyc, s, r4, f4);
    if (rc == OBEM_OK) {
        out[0] = 2.0 * f0 / 1e12;     // FP32 TFLOP/s of packed FMA chains (2 flops per lane-op)
        out[1] = r0;                  // FP32 lane-ops per SM per clock
        out[2] = r1;                  // rsqrt per SM per clock
        out[3] = r2;                  // FP32 lane-ops per SM per clock in the 12:1 mix with rsqrt
        out[4] = f0 / (r0 * sms) / 1e6;   // SM clock during the FMA run, MHz
        out[5] = r3;                  // FP32 lane-ops per SM per clock in the 16:1 mix with rsqrt
        out[6] = r4;                  // FP32 lane-ops per SM per clock in the 14:1 mix with rsqrt
    }
    free(hcyc);
    cudaFree(sink);
    cudaFree(cyc);
    return rc;
}
