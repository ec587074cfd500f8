// BF16 tensor-core GEMM for the trailing updates of the BEM LU factorisation
// (Sec. 2.2, Eq. (matrixBEM): the dense system is the one real dense
// contraction of the method).
//
//   C[M x N] -= A[M x K] B[K x N]      C, A, B: FP32 row-major sub-blocks
//
// The operands are rounded to BF16 (round to nearest even) into K-major
// scratch (A as is, B transposed), then one CTA per 256 x 256 tile of C (tiles
// ordered in groups of 8 row tiles for L2 reuse) runs
// a TMA -> shared memory -> tcgen05.mma pipeline:
//   warp 0, one lane   TMA producer: 64-wide K slices of A (256 rows) and B
//                      (256 rows) into a 3-stage ring, 128B-swizzled
//   warp 1, one lane   MMA issuer: per slice 4 K steps x 2 tcgen05.mma.kind::f16
//                      (M 128, N 256, K 16), one per half of the tile's rows,
//                      both on the stage's B; FP32 accumulation in tensor
//                      memory (two accumulators of 256 columns x 128 lanes: all
//                      512 columns); tcgen05.commit frees a stage
//   warps 0-3          epilogue: tcgen05.ld of their 32 lanes of each
//                      accumulator, through shared memory, C -= D with
//                      coalesced row accesses
// The 256-row tile halves the operand bytes each SM fetches per flop against
// a 128-row one (the 128 x 256 tiles kept the tensor pipe about half busy,
// fed from L2).
// Every wait on an mbarrier is bounded; a wait that runs out records
// OBEM_ERR_TIMEOUT in *err, the kernel lets its issued copies and MMAs finish
// (bounded again), frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "obem_internal.cuh"

namespace {
constexpr int TC_MM = 128;                                        // rows of one MMA and of one accumulator
constexpr int TC_BM = 256, TC_BN = 256, TC_BK = 64, TC_STAGES = 3, TC_THREADS = 128;
constexpr int TC_ACC = TC_BM / TC_MM;                             // accumulators per tile
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;               // 32 KB
constexpr uint32_t TC_B_BYTES = TC_BN * TC_BK * 2;               // 32 KB
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr uint32_t TC_TMEM_COLS = TC_ACC * TC_BN;                 // 512: all of the SM's tensor memory
constexpr int TC_GROUP_M = 8;                                    // row tiles per rasterisation group
constexpr size_t TC_SMEM = 1024 + (size_t)TC_STAGES * TC_STAGE_BYTES + 256;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // 2 s per wait
// instruction descriptor of tcgen05.mma.kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_MM >> 4) << 24);
}

__device__ __forceinline__ uint32_t tc_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void tc_mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ unsigned long long tc_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true once the phase of the given parity has completed; false when it has
// not completed within TC_WAIT_NS of the first poll
__device__ __forceinline__ bool tc_mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = tc_smem(bar);
    const unsigned long long t0 = tc_now();
    for (unsigned i = 0;; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if ((i & 255u) == 255u && tc_now() - t0 > TC_WAIT_NS) return false;
    }
}

__device__ __forceinline__ void tc_tma_load(const CUtensorMap *tm, uint64_t *bar, void *dst, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
                 ::"r"(tc_smem(dst)), "l"((unsigned long long)tm), "r"(tc_smem(bar)), "r"(x), "r"(y)
                 : "memory");
}

// shared-memory matrix descriptor of a K-major, 128B-swizzled operand tile
// (rows of 64 BF16 = 128 bytes, 8-row groups 1024 bytes apart): start
// address >> 4 (bits 0-13), leading offset 1 (unused with this swizzle),
// stride offset 1024 >> 4 (bits 32-45), descriptor version 1 (bit 46),
// swizzle mode 2 = 128B (bits 61-63)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %3, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(accumulate), "r"(TC_IDESC)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of the warp's 32 lanes (thread t: lane t)
__device__ __forceinline__ void tc_tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float *__restrict__ C,
               long long ldc, int M, int N, int K, int *err)
{
    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;
    uint8_t *sB = sm + TC_STAGES * TC_A_BYTES;
    uint64_t *full = (uint64_t *)(sm + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *done = empty + TC_STAGES;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    int *s_fail = (int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile of this CTA: groups of TC_GROUP_M row tiles are walked down the
    // rows first, so the CTAs resident at one time cover a compact block of C
    // and share their A and B slices in L2
    int m_tile, n_tile;
    {
        const int num_m = (M + TC_BM - 1) / TC_BM, num_n = (N + TC_BN - 1) / TC_BN;
        const int pid = blockIdx.x;
        const int per_group = TC_GROUP_M * num_n;
        const int first_m = (pid / per_group) * TC_GROUP_M;
        const int gm = min(num_m - first_m, TC_GROUP_M);
        m_tile = first_m + (pid % per_group) % gm;
        n_tile = (pid % per_group) / gm;
    }
    const int n0 = n_tile * TC_BN, m0 = m_tile * TC_BM;
    const int nk = (K + TC_BK - 1) / TC_BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            tc_mbar_init(&full[s], 1);
            tc_mbar_init(&empty[s], 1);
        }
        tc_mbar_init(done, 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= 2) {
        // the epilogue reads and rewrites this CTA's tile of C: bring it into
        // L2 while the main loop runs (8 lines of 128 bytes per row)
        for (int e = threadIdx.x - 64; e < TC_BM * (TC_BN / 32); e += 64) {
            const int r = m0 + e / (TC_BN / 32), cc = n0 + (e % (TC_BN / 32)) * 32;
            if (r < M && cc < N)
                asm volatile("prefetch.global.L2 [%0];" ::"l"((unsigned long long)(C + (size_t)r * ldc + cc)));
        }
    }
    if (warp == 0 && lane == 0) {
        // producer
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % TC_STAGES;
            if (kb >= TC_STAGES && !tc_mbar_wait(&empty[s], ((kb / TC_STAGES) - 1) & 1)) {
                atomicExch(s_fail, 1);
                break;
            }
            tc_mbar_expect_tx(&full[s], TC_STAGE_BYTES);
            tc_tma_load(&tmA, &full[s], sA + s * TC_A_BYTES, kb * TC_BK, m0);
            tc_tma_load(&tmB, &full[s], sB + s * TC_B_BYTES, kb * TC_BK, n0);
        }
        if (*(volatile int *)s_fail) {
            // let the copies this thread issued land before the CTA exits
            for (int q = kb - 1; q >= 0 && q >= kb - TC_STAGES; --q)
                tc_mbar_wait(&full[q % TC_STAGES], (q / TC_STAGES) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TC_STAGES;
            if (!tc_mbar_wait(&full[s], (kb / TC_STAGES) & 1)) {
                atomicExch(s_fail, 1);
                break;
            }
            tc_fence_after();
            const uint32_t a0 = tc_smem(sA + s * TC_A_BYTES), b0 = tc_smem(sB + s * TC_B_BYTES);
            // accumulator a: rows a*128 .. a*128+127 of the tile (their A rows
            // start a*128 rows = 16 KB into the stage, a whole number of
            // 1024-byte swizzle atoms) in tensor-memory columns a*256 ..;
            // both share the stage's B.  A half of the tile past M is skipped.
#pragma unroll
            for (int j = 0; j < TC_BK / 16; ++j)
#pragma unroll
                for (int a = 0; a < TC_ACC; ++a)
                    if (a == 0 || m0 + a * TC_MM < M)
                        tc_mma(tmem + (uint32_t)(a * TC_BN), tc_desc(a0 + (uint32_t)(a * TC_MM * 128) + 32 * j),
                               tc_desc(b0 + 32 * j), (kb | j) != 0);
            tc_commit(&empty[s]);
        }
        // arrives once every MMA issued above has completed (also on failure)
        tc_commit(done);
    }
    __syncwarp();

    // epilogue: warp w owns accumulator lanes (rows) 32 w .. 32 w + 31
    const bool fine = tc_mbar_wait(done, 0);
    tc_fence_after();
    __syncthreads();
    if (fine && !*(volatile int *)s_fail) {
        float *stage = (float *)sA + warp * 32 * 33;       // pipeline smem is idle now
        for (int acc = 0; acc < TC_ACC; ++acc) {
            const int rbase = m0 + acc * TC_MM + warp * 32;
            if (rbase >= M) break;                          // warp-uniform
            const int nrow = min(32, M - rbase);
            // the 32 rows' values of this lane's column, chunk by chunk of 32
            // columns; the next chunk's loads are in flight while this one is
            // written back
            float vn[32];
            {
                const int col = n0 + lane;
                const float *cp = C + (size_t)rbase * ldc + col;
#pragma unroll
                for (int i = 0; i < 32; ++i) vn[i] = (i < nrow && col < N) ? __ldcg(cp + (size_t)i * ldc) : 0.f;
            }
            for (int c = 0; c < TC_BN; c += 32) {
                if (n0 + c >= N) break;                     // warp-uniform
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = vn[i];
                if (c + 32 < TC_BN && n0 + c + 32 < N) {
                    const int coln = n0 + c + 32 + lane;
                    const float *cpn = C + (size_t)rbase * ldc + coln;
#pragma unroll
                    for (int i = 0; i < 32; ++i) vn[i] = (i < nrow && coln < N) ? __ldcg(cpn + (size_t)i * ldc) : 0.f;
                }
                uint32_t r[32];
                tc_tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * TC_BN + c), r);
#pragma unroll
                for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
                __syncwarp();
                const int col = n0 + c + lane;
                float *cp = C + (size_t)rbase * ldc + col;
                if (col < N) {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (i < nrow) __stcg(cp + (size_t)i * ldc, v[i] - stage[i * 33 + lane]);
                }
                __syncwarp();
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, OBEM_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
}

// out[i * ldo + k] = bf16(A[i * lda + k]), i < M, k < K: blockDim.x threads
// across a row (a multiple of 32, not above K's), blockDim.y rows per pass,
// grid-stride in both
__global__ void tc_cvt_rows_kernel(const float *__restrict__ A, long long lda, int M, int K,
                                   __nv_bfloat16 *__restrict__ out, int ldo)
{
    for (int i = blockIdx.y * blockDim.y + threadIdx.y; i < M; i += gridDim.y * blockDim.y)
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
            out[(size_t)i * ldo + k] = __float2bfloat16_rn(A[(size_t)i * lda + k]);
}

// out[j * ldo + k] = bf16(B[k * ldb + j]), j < N, k < K (transpose through
// a 32 x 32 shared tile: both sides coalesced)
__global__ void tc_cvt_trans_kernel(const float *__restrict__ B, long long ldb, int K, int N,
                                    __nv_bfloat16 *__restrict__ out, int ldo)
{
    __shared__ float t[32][33];
    const int j0 = blockIdx.x * 32;
    for (int k0 = blockIdx.y * 32; k0 < K; k0 += gridDim.y * 32) {
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int k = k0 + r, j = j0 + threadIdx.x;
            t[r][threadIdx.x] = (k < K && j < N) ? B[(size_t)k * ldb + j] : 0.f;
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int j = j0 + r, k = k0 + threadIdx.x;
            if (j < N && k < K) out[(size_t)j * ldo + k] = __float2bfloat16_rn(t[threadIdx.x][r]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*tc_encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static tc_encode_fn tc_encoder()
{
    static tc_encode_fn fn = NULL;
    if (!fn) {
        void *p = NULL;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (tc_encode_fn)p;
    }
    return fn;
}

// 2-D map of a K-major BF16 matrix [rows][ld] with K valid columns, boxes of
// 64 x box_rows, 128-byte swizzle, zero fill outside
static int tc_map(obem_ctx *c, CUtensorMap *m, const void *base, int rows, int K, int ld, int box_rows)
{
    tc_encode_fn enc = tc_encoder();
    if (!enc) return obem_fail(c, OBEM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return obem_fail(c, OBEM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return OBEM_OK;
}

// BF16 scratch of the context for operands up to a_elems / b_elems elements
int obem_tc_reserve(obem_ctx *c, size_t a_elems, size_t b_elems)
{
    if (a_elems * 2 > c->tc_a_bytes) {
        if (c->tc_a) cudaFree(c->tc_a);
        c->tc_a = NULL;
        c->tc_a_bytes = 0;
        OBEM_CUDA(c, cudaMalloc(&c->tc_a, a_elems * 2));
        c->tc_a_bytes = a_elems * 2;
    }
    if (b_elems * 2 > c->tc_b_bytes) {
        if (c->tc_b) cudaFree(c->tc_b);
        c->tc_b = NULL;
        c->tc_b_bytes = 0;
        OBEM_CUDA(c, cudaMalloc(&c->tc_b, b_elems * 2));
        c->tc_b_bytes = b_elems * 2;
    }
    return OBEM_OK;
}

void obem_tc_free(obem_ctx *c)
{
    if (c->tc_a) cudaFree(c->tc_a);
    if (c->tc_b) cudaFree(c->tc_b);
    c->tc_a = c->tc_b = NULL;
    c->tc_a_bytes = c->tc_b_bytes = 0;
}

// C[M x N] -= A[M x K] B[K x N] with BF16 operands and FP32 accumulation;
// C, A, B are FP32 row-major blocks with leading dimensions ldc, lda, ldb.
// Uses the context's BF16 scratch (obem_tc_reserve grows it); err: device
// int receiving OBEM_ERR_TIMEOUT if a bounded wait ran out.
int obem_tc_gemm_sub(obem_ctx *c, float *C, long long ldc, const float *A, long long lda, const float *B, long long ldb,
                     int M, int N, int K, int *err, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return OBEM_OK;
    const int ldk = (K + 7) / 8 * 8;                       // 16-byte row pitch for the tensor maps
    int rc = obem_tc_reserve(c, (size_t)M * ldk, (size_t)N * ldk);
    if (rc != OBEM_OK) return rc;
    __nv_bfloat16 *Ab = (__nv_bfloat16 *)c->tc_a, *Bb = (__nv_bfloat16 *)c->tc_b;
    {
        // skinny operands (K of 64 against tall M) get several rows per block
        const int tx = K >= 256 ? 256 : (K + 31) / 32 * 32, ty = 256 / tx;
        const int gx = K >= 256 ? ((K + 255) / 256 < 64 ? (K + 255) / 256 : 64) : 1;
        const int gyn = (M + ty - 1) / ty, gy = gyn < 4096 ? gyn : 4096;
        tc_cvt_rows_kernel<<<dim3(gx, gy), dim3(tx, ty), 0, s>>>(A, lda, M, K, Ab, ldk);
        dim3 gt((N + 31) / 32, (K + 31) / 32 < 65535 ? (K + 31) / 32 : 65535);
        tc_cvt_trans_kernel<<<gt, dim3(32, 8), 0, s>>>(B, ldb, K, N, Bb, ldk);
        OBEM_LAUNCH(c);
    }
    CUtensorMap ma, mb;
    rc = tc_map(c, &ma, Ab, M, K, ldk, TC_BM);
    if (rc == OBEM_OK) rc = tc_map(c, &mb, Bb, N, K, ldk, TC_BN);
    if (rc != OBEM_OK) return rc;
    static unsigned long long attr = 0;   // devices done (a bit each)
    if (!(attr >> (c->device & 63) & 1ull)) {
        OBEM_CUDA(c, cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        attr |= 1ull << (c->device & 63);
    }
    const long long tiles = (long long)((N + TC_BN - 1) / TC_BN) * ((M + TC_BM - 1) / TC_BM);
    if (tiles > 0x7fffffffll) return obem_fail(c, OBEM_ERR_ARG, "tensor-core GEMM: %d x %d exceeds the grid", M, N);
    tc_gemm_kernel<<<(unsigned)tiles, TC_THREADS, TC_SMEM, s>>>(ma, mb, C, ldc, M, N, K, err);
    OBEM_LAUNCH(c);
    return OBEM_OK;
}

// C ABI hook: the same update on caller arrays (FP32, row-major), for tests
// and measurement of the tensor-core path; synchronises the stream and
// reports a bounded-wait timeout as OBEM_ERR_TIMEOUT.
extern "C" int obem_tc_gemm(obem_ctx *c, float *C, int64_t ldc, const float *A, int64_t lda, const float *B,
                            int64_t ldb, int32_t M, int32_t N, int32_t K, obem_stream stream)
{
    if (!c || !C || !A || !B) return OBEM_ERR_ARG;
    if (M < 0 || N < 0 || K < 0 || ldc < N || lda < K || ldb < N) return obem_fail(c, OBEM_ERR_ARG, "tc_gemm: bad sizes");
    cudaStream_t s = (cudaStream_t)stream;
    int *err = NULL;
    OBEM_CUDA(c, cudaMalloc((void **)&err, sizeof(int)));
    int h = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    int rc = OBEM_OK;
    if (e == cudaSuccess) rc = obem_tc_gemm_sub(c, C, ldc, A, lda, B, ldb, M, N, K, err, s);
    if (e == cudaSuccess && rc == OBEM_OK) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && rc == OBEM_OK) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (rc != OBEM_OK) return rc;
    if (e != cudaSuccess) return obem_fail(c, OBEM_ERR_CUDA, "tc_gemm: %s", cudaGetErrorString(e));
    if (h != 0) return obem_fail(c, OBEM_ERR_TIMEOUT, "tc_gemm: a bounded wait ran out");
    return OBEM_OK;
}
