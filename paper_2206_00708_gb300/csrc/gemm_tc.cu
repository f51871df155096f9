// Multi-column MTF products on the 5th-generation tensor cores (tcgen05), for the
// batched right-hand sides of the mixed-precision mode (paper eq. mtf:discrete; the
// dense products are the a9 step of the solve, Sec. 3.3 / Sec. 5.1).
//
// A block row b of the MTF is z_b = c1 A1 x1 + c2 A2 x2 with complex64 matrices A
// (N_b x N_b, row-major) and R complex right-hand sides.  Stored as interleaved
// (re, im) floats, one row of [A1 | A2] is a real K-vector of length K_b = 4 N_b, and
//     Re z = sum_k A[k] B[r][k],   Im z = sum_k A[k] B[R + r][k]
// with, for the entry j of x (x = x1 for k < 2 N_b, x2 after, scaled by c):
//     B[r][2j] = c Re x_j,  B[r][2j+1] = -c Im x_j,  B[R+r][2j] = c Im x_j,  B[R+r][2j+1] = c Re x_j.
// So each block row is one real GEMM  Z (N_b x 2R) = A (N_b x K_b) B^T, with A read
// in place (K-major) and B (2R x K_b, K-major) built per product.
//
// Precision: kind::tf32 (10-bit mantissa) with a three-term split: A = Ah + Al and
// B = Bh + Bl with Ah, Bh rounded to TF32 and Al, Bl the (exact) FP32 remainders;
// Z = Ah Bh + Ah Bl + Al Bh, accumulated in FP32 in tensor memory (the dropped Al Bl
// is below 2^-22 relative).  This is an inner-solver product: the refinement's
// outer residual is computed in FP64 on the stored complex64 matrices.
//
// One CTA per 128-row tile of a block row, 256 threads.  Per K stage of 32 floats all
// threads stage A (split into Ah, Al) and copy Bh, Bl into shared memory in the
// canonical no-swizzle K-major layout (core matrices of 8 rows x 16 bytes); one
// thread issues 4 x 3 MMAs (M = 128, N = 2R, K = 8) into one of 2-8 TMEM accumulators
// (chosen by stage, summed in FP32 at the end) and commits them to the stage's
// mbarrier; two shared-memory stages alternate and the global loads of A for stages
// s + 1 and s + 2 are in flight (two register buffers) while stage s is staged and
// issued.  With fewer row tiles than SMs (or as the autotuner chose for the shape)
// the K range is split between two CTAs whose results are added into a zeroed z
// (two addends: their order cannot change the sum).  The epilogue reads the
// accumulators with tcgen05.ld (warps 0-3: real parts, warps 4-7: imaginary parts).
#include "bem_internal.cuh"

#include <algorithm>

namespace bem {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;       // rows per CTA (MMA M)
constexpr int TC_KS = 32;       // K floats per stage (4 MMAs of K = 8)
constexpr int TC_A_SUB = 4096;  // bytes of one 128 x 8 A sub-tile
constexpr int TC_A_STAGE = 4 * TC_A_SUB;
constexpr long long TC_WAIT_LIMIT = 1ll << 26;  // mbarrier polls before giving up (seconds)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, K-major; leading (K-direction)
// core-matrix stride 128 bytes, stride (row-group direction) 256 bytes
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    const uint64_t start = (addr >> 4) & 0x3FFFull;
    const uint64_t lbo = (128u >> 4) & 0x3FFFull;
    const uint64_t sbo = (256u >> 4) & 0x3FFFull;
    return start | (lbo << 16) | (sbo << 32) | (1ull << 46);  // version 1, base offset 0, layout 0
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = n, M = 128
__device__ __forceinline__ uint32_t instr_desc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait for the completion of the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// the double of a float built from its bits with integer operations (zero and FP32
// subnormals give 0, infinities and NaNs stay so)
__device__ __forceinline__ double widen_f32(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const uint64_t de = e == 0xFFu ? 0x7FFull : (uint64_t)(e + 896u);
    return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | (de << 52) |
                                            ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// round to the nearest TF32 value (10 explicit mantissa bits); finite inputs
__device__ __forceinline__ float tf32_rn(float a) {
    return __uint_as_float((__float_as_uint(a) + 0x1000u) & 0xFFFFE000u);
}

// byte offset of element (row, kk) (kk < 32) in a stage tile with `rows` rows,
// stored as 4 sub-tiles of K = 8 in the canonical layout
__host__ __device__ __forceinline__ uint32_t tile_off(int row, int kk, int rows) {
    const int k8 = kk >> 3, c = (kk >> 2) & 1, e = kk & 3;
    return (uint32_t)(k8 * rows * 32 + (row >> 3) * 256 + c * 128 + (row & 7) * 16 + e * 4);
}

struct TcBlockRow {
    const float* a1;  // complex64 matrices as interleaved floats, row-major
    const float* a2;
    const float* bh;  // B stages (hi / lo) of this block row
    const float* bl;
    int64_t N, base;  // order and first row of the block row in z
    int stages;       // ceil(4 N / 32)
    int tiles;        // ceil(N / 128)
};

struct TcArgs {
    TcBlockRow br[4];
    int R;       // right-hand sides (columns of z written)
    int RP;      // padded to a multiple of 8; MMA N = 2 RP
    int64_t n;   // z column length
};

// B stages of all four block rows from x (R columns of n complex values)
struct TcPrep {
    float* bh[4];
    float* bl[4];
    int64_t N[4], x1[4], x2[4];
    double c1[4], c2[4];
    int stages[4];
    int R, RP;
    int64_t n;
};

__global__ void k_tc_prep(TcPrep P, const double2* __restrict__ x) {
    const int b = blockIdx.y;
    const int rows = 2 * P.RP;
    const int64_t per_stage = (int64_t)rows * TC_KS;
    const int64_t total = per_stage * P.stages[b];
    const int64_t N = P.N[b];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / per_stage;
        const int rem = (int)(t - s * per_stage);
        const int row = rem / TC_KS, kk = rem % TC_KS;
        const int64_t k = s * TC_KS + kk;
        const int r = row < P.RP ? row : row - P.RP;
        const bool imag_row = row >= P.RP;
        float v = 0.0f;
        if (r < P.R && k < 4 * N) {
            const bool second = k >= 2 * N;
            const int64_t j = (second ? k - 2 * N : k) >> 1;
            const int part = (int)(k & 1);
            const double c = second ? P.c2[b] : P.c1[b];
            const double2 xv = x[(int64_t)r * P.n + (second ? P.x2[b] : P.x1[b]) + j];
            const double val = imag_row ? (part == 0 ? xv.y : xv.x) : (part == 0 ? xv.x : -xv.y);
            v = (float)(c * val);
        }
        const float h = tf32_rn(v);
        const int64_t off = s * (per_stage * 4) + tile_off(row, kk, rows);  // bytes
        *reinterpret_cast<float*>(reinterpret_cast<char*>(P.bh[b]) + off) = h;
        *reinterpret_cast<float*>(reinterpret_cast<char*>(P.bl[b]) + off) = v - h;
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc(TcArgs P, double* __restrict__ z, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_fail;

    // which block row and row tile
    int b = 0, tile = blockIdx.x;
    while (b < 3 && tile >= P.br[b].tiles) {
        tile -= P.br[b].tiles;
        ++b;
    }
    const TcBlockRow& br = P.br[b];  // (kernel parameter space)
    const float* __restrict__ a1 = br.a1;
    const float* __restrict__ a2 = br.a2;
    const int64_t N = br.N;
    // K split: blockIdx.y of gridDim.y takes stages [s_begin, s_end)
    const int s_begin = (int)((int64_t)br.stages * blockIdx.y / gridDim.y);
    const int s_end = (int)((int64_t)br.stages * (blockIdx.y + 1) / gridDim.y);
    const int S = s_end - s_begin;
    const int nb = 2 * P.RP;                 // MMA N and B rows
    const int b_stage = nb * TC_KS * 4;      // bytes of one B stage (hi or lo)
    const int stage_bytes = 2 * TC_A_STAGE + 2 * b_stage;
    // stage s accumulates into accumulator s % nacc (columns [acc nb, acc nb + nb)):
    // the tensor cores' FP32 accumulation is biased, and nacc shorter chains, summed
    // at the end, keep its error near 1e-6 over K = 4 N
    const int nacc = nb <= 64 ? 8 : nb <= 128 ? 4 : 2;
    const int used = nacc * nb;
    const int ncols = used <= 32 ? 32 : used <= 64 ? 64 : used <= 128 ? 128 : used <= 256 ? 256 : 512;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // visible to the async proxy
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint32_t idesc = instr_desc(nb);

    // A staging assignment: thread -> (row, half of the 32 K floats)
    const int arow = threadIdx.x >> 1, ahalf = threadIdx.x & 1;
    const int64_t grow = (int64_t)tile * TC_M + arow;  // row within the block row
    const bool row_ok = grow < N;

    // A is loaded into registers two stages ahead (two register buffers, used
    // alternately), so two stages of global loads are in flight while a stage is
    // staged and its MMAs are issued
    auto load_a = [&](float2 (&pa)[8], int sg) {
        const int64_t k0 = (int64_t)sg * TC_KS + ahalf * 16;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t k = k0 + 2 * q;
            float2 v = make_float2(0.f, 0.f);
            if (row_ok) {
                if (k < 2 * N) v = *reinterpret_cast<const float2*>(a1 + grow * 2 * N + k);
                else if (k < 4 * N) v = *reinterpret_cast<const float2*>(a2 + grow * 2 * N + (k - 2 * N));
            }
            pa[q] = v;
        }
    };
    float2 pa0[8], pa1[8];
    if (S > 0) load_a(pa0, s_begin);
    if (S > 1) load_a(pa1, s_begin + 1);
    auto stage = [&](float2 (&pa)[8], int ls) {
        const int sg = s_begin + ls;  // global stage
        const int buf = ls & 1;
        unsigned char* st = tsm + buf * stage_bytes;
        if (ls >= 2) {  // MMAs of stage ls - 2 read this buffer
            if (!mbar_wait(smem_u32(&mbar[buf]), (uint32_t)(((ls - 2) >> 1) & 1))) s_fail = 1;
        }
        // A: 16 floats per thread, split into TF32 hi / lo
#pragma unroll
        for (int g4 = 0; g4 < 4; ++g4) {
            const int kk = ahalf * 16 + 4 * g4;
            const float a0 = pa[2 * g4].x, a1v = pa[2 * g4].y, a2v = pa[2 * g4 + 1].x, a3 = pa[2 * g4 + 1].y;
            float4 h, l;
            h.x = tf32_rn(a0); l.x = a0 - h.x;
            h.y = tf32_rn(a1v); l.y = a1v - h.y;
            h.z = tf32_rn(a2v); l.z = a2v - h.z;
            h.w = tf32_rn(a3); l.w = a3 - h.w;
            const uint32_t off = tile_off(arow, kk, TC_M);
            *reinterpret_cast<float4*>(st + off) = h;
            *reinterpret_cast<float4*>(st + TC_A_STAGE + off) = l;
        }
        if (ls + 2 < S) load_a(pa, sg + 2);
        // B: contiguous copies of the prepared stage tiles
        {
            const float4* __restrict__ sh = reinterpret_cast<const float4*>(
                reinterpret_cast<const char*>(br.bh) + (int64_t)sg * b_stage);
            const float4* __restrict__ sl = reinterpret_cast<const float4*>(
                reinterpret_cast<const char*>(br.bl) + (int64_t)sg * b_stage);
            float4* dh = reinterpret_cast<float4*>(st + 2 * TC_A_STAGE);
            float4* dl = reinterpret_cast<float4*>(st + 2 * TC_A_STAGE + b_stage);
            for (int i = threadIdx.x; i < b_stage / 16; i += TC_THREADS) {
                dh[i] = sh[i];
                dl[i] = sl[i];
            }
        }
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(st), al = ah + TC_A_STAGE;
            const uint32_t bh = ah + 2 * TC_A_STAGE, bl = bh + b_stage;
#pragma unroll
            for (int k8 = 0; k8 < 4; ++k8) {
                const uint64_t dah = smem_desc(ah + k8 * TC_A_SUB), dal = smem_desc(al + k8 * TC_A_SUB);
                const uint64_t dbh = smem_desc(bh + k8 * nb * 32), dbl = smem_desc(bl + k8 * nb * 32);
                const uint32_t d = tmem + (uint32_t)((ls % nacc) * nb);
                mma_tf32(d, dah, dbh, idesc, (ls >= nacc || k8 > 0) ? 1 : 0);
                mma_tf32(d, dah, dbl, idesc, 1);
                mma_tf32(d, dal, dbh, idesc, 1);
            }
            mma_commit(smem_u32(&mbar[buf]));
        }
    };
    for (int ls = 0; ls < S; ls += 2) {
        stage(pa0, ls);
        if (ls + 1 < S) stage(pa1, ls + 1);
    }
    // the last commit covers every MMA issued before it
    if (S > 0 && !mbar_wait(smem_u32(&mbar[(S - 1) & 1]), (uint32_t)(((S - 1) >> 1) & 1))) s_fail = 1;
    tc_fence_after();
    __syncthreads();
    if (!s_fail) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns [h RP, h RP + RP), h = w / 4;
        // the accumulators are summed in FP32 and widened to FP64 with integer operations
        // (GB300's FP64 pipe runs at 1/64 of the FP32 rate: FP64 sums here cost as much as the MMAs)
        const int q = warp & 3, h = warp >> 2;
        const int64_t row = (int64_t)tile * TC_M + 32 * q + lane;
        for (int c0 = 0; c0 < P.RP; c0 += 8) {
            float sum[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int acc = 0; acc < nacc && acc < S; ++acc) {  // accumulators this CTA wrote
                uint32_t v[8];
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * nb + h * P.RP + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                    "tcgen05.wait::ld.sync.aligned;"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                    : "r"(taddr)
                    : "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) sum[j] += __uint_as_float(v[j]);
            }
            if (row < N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int r = c0 + j;
                    if (r >= P.R) continue;
                    double* zz = z + 2 * ((int64_t)r * P.n + br.base + row) + h;
                    if (gridDim.y == 1) *zz = widen_f32(sum[j]);
                    else atomicAdd(zz, widen_f32(sum[j]));  // two K halves into a zeroed z: order-free
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

int tc_padded_columns(int R) { return (R + 7) / 8 * 8; }

size_t tc_workspace_bytes(const int64_t N[4], int RP) {
    size_t total = 0;
    for (int b = 0; b < 4; ++b) {
        const int64_t stages = (4 * N[b] + TC_KS - 1) / TC_KS;
        total += 2 * (size_t)stages * (2 * RP) * TC_KS * 4;
    }
    return total;
}

// z (R columns of n, complex128) = the four block rows of the MTF applied to x
// (R columns), complex64 matrices a1[b], a2[b] with coefficients c1[b], c2[b].
bem_status mtf_product_tc(const float2* const a1[4], const float2* const a2[4], const double c1[4],
                          const double c2[4], const int64_t N[4], const int64_t base[4], const int64_t x1[4],
                          const int64_t x2[4], int64_t n, int R, const double2* x, double2* z, void* work,
                          size_t work_bytes, int* err, cudaStream_t s) {
    const int RP = tc_padded_columns(R);
    if (R < 1 || 2 * RP > 256) {
        set_error("tensor-core product: 1 to 128 right-hand sides per call");
        return BEM_E_INVALID_ARG;
    }
    if (work_bytes < tc_workspace_bytes(N, RP)) {
        set_error("tensor-core product: workspace too small");
        return BEM_E_INTERNAL;
    }
    TcPrep pp{};
    TcArgs ta{};
    char* w = static_cast<char*>(work);
    int tiles = 0;
    for (int b = 0; b < 4; ++b) {
        const int stages = (int)((4 * N[b] + TC_KS - 1) / TC_KS);
        const size_t bytes = (size_t)stages * (2 * RP) * TC_KS * 4;
        pp.bh[b] = reinterpret_cast<float*>(w);
        pp.bl[b] = reinterpret_cast<float*>(w + bytes);
        w += 2 * bytes;
        pp.N[b] = N[b];
        pp.x1[b] = x1[b];
        pp.x2[b] = x2[b];
        pp.c1[b] = c1[b];
        pp.c2[b] = c2[b];
        pp.stages[b] = stages;
        TcBlockRow& br = ta.br[b];
        br.a1 = reinterpret_cast<const float*>(a1[b]);
        br.a2 = reinterpret_cast<const float*>(a2[b]);
        br.bh = pp.bh[b];
        br.bl = pp.bl[b];
        br.N = N[b];
        br.base = base[b];
        br.stages = stages;
        br.tiles = (int)((N[b] + TC_M - 1) / TC_M);
        tiles += br.tiles;
    }
    pp.R = R;
    pp.RP = RP;
    pp.n = n;
    ta.R = R;
    ta.RP = RP;
    ta.n = n;
    BEM_LAUNCH(k_tc_prep, dim3(152 * 4, 4), 256, 0, s, pp, x);
    const int b_stage = 2 * RP * TC_KS * 4;
    // at least 116 KB of shared memory: one CTA per SM, so its TMEM allocation (up to
    // all 512 columns) never waits for another CTA
    const int smem = std::max(2 * (2 * TC_A_STAGE + 2 * b_stage), 116 * 1024);
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // fewer row tiles than SMs: split K in two halves (their two sums commute exactly),
    // unless the autotuner measured otherwise for this shape
    int sms = 0, dev = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ksplit = tune_get(TUNE_GEMM_TC, RP, n, TuneChoice{0, tiles < sms ? 2 : 1, 0.0}).variant;
    if (ksplit > 1) BEM_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)R * n * sizeof(double2), s));
    BEM_LAUNCH(k_gemm_tc, dim3(tiles, ksplit), TC_THREADS, smem, s, ta, reinterpret_cast<double*>(z), err);
    return BEM_OK;
}

}  // namespace bem
