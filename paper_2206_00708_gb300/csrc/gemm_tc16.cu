// Multi-column MTF products on the tcgen05 tensor cores with an FP16 (or BF16) two-term
// split of both operands, fed by TMA: the split-complex tensor-core variants of the
// mixed-precision mode (paper eq. mtf:discrete; the dense products are the a9 step of
// the solve, Sec. 3.3 / Sec. 5.1).  BF16 keeps 8 + 8 significant bits per operand
// (products to ~2^-16) against FP16's 11 + 11 (~2^-22), in the same kernel.
//
// A block row b of the MTF is z_b = c1 A1 x1 + c2 A2 x2 with complex64 N_b x N_b
// matrices A.  As in the TF32 product, one row of [A1 | A2] read as interleaved
// (re, im) floats is a real K-vector (K = 4 N_b), and Re z, Im z of R right-hand sides
// are one real GEMM  Z (N_b x 2R) = A (N_b x K) B^T  with B built from x (rows r < RP:
// (c Re x_j, -c Im x_j) pairs; rows RP + r: (c Im x_j, c Re x_j)).
//
// Split.  Each block row keeps an operator copy A 2^eA = Ah + Al with Ah = fp16(A 2^eA)
// and Al = fp16(A 2^eA - Ah) (22 significant bits together), the power of two 2^eA
// putting the largest |entry| of the block row below 2^14 (FP16's largest finite value
// is 65504); rows are padded with zeros to Kp = 64 * ceil(K / 64) halves (a multiple of
// 128 bytes).  B is split the same way per product, with a power
// of two per (block row, column) from the largest |c x_r|.  The tensor cores form
// Ah Bh + Ah Bl + Al Bh (the dropped Al Bl is below 2^-22 relative) in FP32; the
// epilogue scales by 2^-(eA + eB).  The operator copy has 8 bytes per complex entry,
// as much as the complex64 copy it replaces, and FP16 MMAs run at twice the TF32 rate.
//
// Layout.  Both copies are stored pre-tiled in the order the kernel reads them, each
// tile already in the tensor cores' 128-byte-swizzled K-major shared-memory layout
// (byte a of a tile at a ^ ((a >> 7 & 7) << 4): rows of 128 bytes, the 16-byte chunk
// index XORed with the row within its group of 8): the operator as [row tile of 128
// rows][stage of 64 halves] tiles of 16 KB, B as [stage] tiles of 2 RP rows.  A stage
// is then a few contiguous TMA bulk copies (the tile product's access pattern, which
// streams at HBM rate), instead of 128 separate 128-byte row pieces.
//
// Pipeline (one CTA per 128-row tile of a block row and K range; 192 threads): warp 0
// lane 0 issues the bulk copies of each stage (Ah, Al: 16 KB each; Bh, Bl: 2 RP x 128
// bytes each) into a ring of 2-4 shared-memory buffers (full barriers: transaction
// bytes; empty barriers: tcgen05.commit); warp 1 lane 0 issues 4 K-steps x 3 MMAs
// (M 128, N 2 RP, K 16) per stage into one of 2-8 TMEM accumulators chosen by stage
// (the tensor cores' FP32 accumulation is biased over long chains; shorter chains keep
// it near 1e-7); warps 2-5 read the accumulators with tcgen05.ld, sum them in FP32 and
// write z.  Every mbarrier wait is bounded; a wait that gives up sets the error flag,
// and the CTA still drains its copies and frees its TMEM.
#include "bem_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

namespace bem {

namespace {

// the 16-bit operand type: FP16 (11 significant bits, range handled by the scaling) or
// BF16 (8 significant bits, FP32's range); its tcgen05 instruction-descriptor format code
struct F16 {
    __device__ static uint16_t from(float x) { return __half_as_ushort(__float2half_rn(x)); }
    __device__ static float to(uint16_t b) { return __half2float(__ushort_as_half(b)); }
    static constexpr uint32_t FMT = 0;
};
struct BF16 {
    __device__ static uint16_t from(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
    __device__ static float to(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
    static constexpr uint32_t FMT = 1;
};
// a 16-bit pair (low half first in memory)
__device__ __forceinline__ uint32_t pack16(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

constexpr int T16_THREADS = 192;
constexpr int T16_M = 128;                    // rows per CTA (MMA M)
constexpr int T16_KS = 64;                    // K halves per stage (128 bytes per row)
constexpr int T16_A_PART = T16_M * T16_KS * 2;  // bytes of Ah or Al of one stage (16 KB)
constexpr long long T16_WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes
// apart (rows of 128 bytes), version 1 (tcgen05)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    const uint64_t start = (addr >> 4) & 0x3FFFull;
    const uint64_t lbo = 1ull;                 // not used by swizzled K-major layouts
    const uint64_t sbo = (1024u >> 4) & 0x3FFFull;
    return start | (lbo << 16) | (sbo << 32) | (1ull << 46) | (2ull << 61);
}

// instruction descriptor: D = F32, A = B = F16 (fmt 0) or BF16 (fmt 1), both K-major,
// N = n, M = 128
__device__ __forceinline__ uint32_t f16_idesc(int n, uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(T16_M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit_to(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// bounded wait for the completion of the phase with the given parity; false on timeout
__device__ __forceinline__ bool bar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < T16_WAIT_LIMIT; ++it) {
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

// one bulk copy global -> shared completing on mbar (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// halves offset of element (row, kk) (kk < 64) in a swizzled tile of 128-byte rows
__host__ __device__ __forceinline__ int64_t swz(int row, int kk) {
    const int a = row * 128 + kk * 2;
    return (a ^ (((a >> 7) & 7) << 4)) >> 1;
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// the double of a float built from its bits with integer operations (zero and FP32
// subnormals give 0, infinities and NaNs stay so)
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const uint64_t de = e == 0xFFu ? 0x7FFull : (uint64_t)(e + 896u);
    return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | (de << 52) |
                                            ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// largest |v| of non-negative floats kept as bit patterns (monotone for v >= 0)
__device__ __forceinline__ void max_bits(int* a, float v) { atomicMax(a, __float_as_int(v)); }

// 2^e that puts m (> 0) below 2^14; 0 for m = 0 or not finite
__host__ __device__ __forceinline__ int top_exponent(float m) {
    if (!(m > 0.0f) || !(m < 3.0e38f)) return 0;
    int ex = 0;
    frexpf(m, &ex);  // m < 2^ex
    return 14 - ex;
}

struct T16Row {
    int64_t N, base;  // order and first row of the block row in z
    int stages;       // Kp / 64
    int tiles;        // ceil(N / 128)
    int eA;           // operator scale exponent
};

struct T16Args {
    const __half* ah[4];  // operator copies, [tile][stage] 16 KB swizzled tiles
    const __half* al[4];
    const __half* bh[4];  // B of this product, [stage] swizzled tiles of 2 RP rows
    const __half* bl[4];
    T16Row br[4];
    const int* eB;  // [4][RP] column scale exponents of this product
    int R, RP;
    int64_t n;      // z column length
    int ksplit;
};

// ---- operator copy: [A1 | A2] rows as (hi, lo) halves, padded to Kp
__global__ void k_t16_absmax(const float* __restrict__ a, int64_t count, int* __restrict__ out) {
    float m = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) max_bits(out, m);
}

template <class TR>
__global__ void k_t16_split_ops(const float* __restrict__ a1, const float* __restrict__ a2, int64_t N, int64_t Kp,
                                float scale, __half* __restrict__ hi, __half* __restrict__ lo) {
    const int64_t total = N * (2 * N);  // complex entries of the row [A1 | A2]
    const int64_t stages = Kp / T16_KS;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / (2 * N), j = t % (2 * N);  // K index k = 2 j
        float2 v = j < N ? *reinterpret_cast<const float2*>(a1 + row * 2 * N + 2 * j)
                         : *reinterpret_cast<const float2*>(a2 + row * 2 * N + 2 * (j - N));
        v.x *= scale;
        v.y *= scale;
        const uint16_t hx = TR::from(v.x), hy = TR::from(v.y);
        const uint16_t lx = TR::from(v.x - TR::to(hx)), ly = TR::from(v.y - TR::to(hy));
        const int64_t k = 2 * j, tile = row / T16_M, st = k / T16_KS;
        const int64_t off = (tile * stages + st) * (T16_M * T16_KS) + swz((int)(row % T16_M), (int)(k % T16_KS));
        *reinterpret_cast<uint32_t*>(hi + off) = pack16(hx, hy);
        *reinterpret_cast<uint32_t*>(lo + off) = pack16(lx, ly);
    }
}

// ---- per product: column maxima, scale exponents, B (hi, lo)
struct T16Prep {
    __half* bh[4];
    __half* bl[4];
    int64_t N[4], Kp[4], x1[4], x2[4];
    double c1[4], c2[4];
    int R, RP;
    int64_t n;
};

__global__ void k_t16_colmax(const double2* __restrict__ x, int64_t n, int R, int* __restrict__ xmax) {
    const int r = blockIdx.y;
    if (r >= R) return;
    float m = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[(int64_t)r * n + i];
        m = fmaxf(m, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) max_bits(&xmax[r], m);
}

__global__ void k_t16_scales(T16Prep P, const int* __restrict__ xmax, int* __restrict__ eB) {
    const int b = blockIdx.x, r = threadIdx.x;
    if (r >= P.RP) return;
    int e = 0;
    if (r < P.R) {
        const float c = (float)fmax(fabs(P.c1[b]), fabs(P.c2[b]));
        e = top_exponent(c * __int_as_float(xmax[r]));
    }
    eB[b * P.RP + r] = e;
}

template <class TR>
__global__ void k_t16_prep(T16Prep P, const double2* __restrict__ x, const int* __restrict__ eB) {
    const int b = blockIdx.z, r = blockIdx.y;
    if (r >= P.R) return;
    const int64_t N = P.N[b];
    const int nb = 2 * P.RP;
    const float s = ldexpf(1.0f, eB[b * P.RP + r]);
    __half* __restrict__ bh = P.bh[b];
    __half* __restrict__ bl = P.bl[b];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < 2 * N; j += (int64_t)gridDim.x * blockDim.x) {
        const bool second = j >= N;
        const double c = second ? P.c2[b] : P.c1[b];
        const double2 xv = x[(int64_t)r * P.n + (second ? P.x2[b] + (j - N) : P.x1[b] + j)];
        const float re = (float)(c * xv.x) * s, im = (float)(c * xv.y) * s;
        // real row: (re, -im); imaginary row: (im, re)
        const uint16_t h_re = TR::from(re), h_im = TR::from(im);
        const uint16_t l_re = TR::from(re - TR::to(h_re)), l_im = TR::from(im - TR::to(h_im));
        const uint16_t nh_im = h_im ^ 0x8000u, nl_im = l_im ^ 0x8000u;  // sign flips (both formats)
        const int64_t k = 2 * j, st = k / T16_KS;
        const int kk = (int)(k % T16_KS);
        const int64_t tbase = st * (int64_t)nb * T16_KS;
        const int64_t ore = tbase + swz(r, kk), oim = tbase + swz(P.RP + r, kk);
        *reinterpret_cast<uint32_t*>(bh + ore) = pack16(h_re, nh_im);
        *reinterpret_cast<uint32_t*>(bl + ore) = pack16(l_re, nl_im);
        *reinterpret_cast<uint32_t*>(bh + oim) = pack16(h_im, h_re);
        *reinterpret_cast<uint32_t*>(bl + oim) = pack16(l_im, l_re);
    }
}

template <class TR>
__global__ void __launch_bounds__(T16_THREADS, 1) k_gemm_tc16(const T16Args P,
                                                               double* __restrict__ z, int* __restrict__ err) {
    extern __shared__ unsigned char t16_raw[];
    __shared__ __align__(8) uint64_t full[4], empty[4], done;
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_fail;

    int b = 0, tile = blockIdx.x;
    while (b < 3 && tile >= P.br[b].tiles) {
        tile -= P.br[b].tiles;
        ++b;
    }
    const T16Row& br = P.br[b];
    const int s_begin = (int)((int64_t)br.stages * blockIdx.y / gridDim.y);
    const int s_end = (int)((int64_t)br.stages * (blockIdx.y + 1) / gridDim.y);
    const int S = s_end - s_begin;
    const int nb = 2 * P.RP;                         // MMA N and B rows
    const int b_part = nb * T16_KS * 2;              // bytes of Bh or Bl of one stage
    const int stage_bytes = 2 * T16_A_PART + 2 * b_part;
    const int NS = stage_bytes <= 48 * 1024 ? 4 : stage_bytes <= 64 * 1024 ? 3 : 2;
    const int nacc = nb <= 64 ? 8 : nb <= 128 ? 4 : 2;
    const int used = nacc * nb;
    const int ncols = used <= 32 ? 32 : used <= 64 ? 64 : used <= 128 ? 128 : used <= 256 ? 256 : 512;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // stage buffers at a 1024-byte boundary (128-byte swizzle atoms)
    const uint32_t raw = smem_addr(t16_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int i = 0; i < NS; ++i) {
            bar_init(smem_addr(&full[i]), 1);
            bar_init(smem_addr(&empty[i]), 1);
        }
        bar_init(smem_addr(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0 && lane == 0) {
        // ---- producer: TMA loads of every stage of this CTA's K range
        int issued = 0;
        for (int ls = 0; ls < S; ++ls) {
            const int buf = ls % NS;
            if (ls >= NS && !bar_wait(smem_addr(&empty[buf]), (uint32_t)((ls / NS - 1) & 1))) {
                s_fail = 1;
                break;
            }
            const uint32_t st = base + (uint32_t)(buf * stage_bytes);
            const uint32_t fb = smem_addr(&full[buf]);
            bar_expect_tx(fb, (uint32_t)stage_bytes);
            const int sg = s_begin + ls;
            const int64_t ao = ((int64_t)tile * br.stages + sg) * (T16_M * T16_KS);  // halves
            const int64_t bo = (int64_t)sg * nb * T16_KS;
            bulk_copy(st, P.ah[b] + ao, (uint32_t)T16_A_PART, fb);
            bulk_copy(st + T16_A_PART, P.al[b] + ao, (uint32_t)T16_A_PART, fb);
            bulk_copy(st + 2 * T16_A_PART, P.bh[b] + bo, (uint32_t)b_part, fb);
            bulk_copy(st + 2 * T16_A_PART + b_part, P.bl[b] + bo, (uint32_t)b_part, fb);
            issued = ls + 1;
        }
        // drain: the last stages issued may still be in flight if the consumer gave up
        for (int t = std::max(0, issued - NS); t < issued; ++t)
            if (!bar_wait(smem_addr(&full[t % NS]), (uint32_t)((t / NS) & 1))) s_fail = 1;
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issue
        const uint32_t idesc = f16_idesc(nb, TR::FMT);
        for (int ls = 0; ls < S; ++ls) {
            const int buf = ls % NS;
            if (!bar_wait(smem_addr(&full[buf]), (uint32_t)((ls / NS) & 1))) {
                s_fail = 1;
                break;
            }
            fence_after();
            const uint32_t st = base + (uint32_t)(buf * stage_bytes);
            const uint32_t d = tmem + (uint32_t)((ls % nacc) * nb);
#pragma unroll
            for (int k = 0; k < T16_KS / 16; ++k) {
                const uint32_t ko = (uint32_t)(k * 32);  // 16 halves along K inside the swizzle atom
                const uint64_t dah = sw128_desc(st + ko), dal = sw128_desc(st + T16_A_PART + ko);
                const uint64_t dbh = sw128_desc(st + 2 * T16_A_PART + ko);
                const uint64_t dbl = sw128_desc(st + 2 * T16_A_PART + b_part + ko);
                mma_f16(d, dah, dbh, idesc, (ls >= nacc || k > 0) ? 1 : 0);
                mma_f16(d, dah, dbl, idesc, 1);
                mma_f16(d, dal, dbh, idesc, 1);
            }
            commit_to(smem_addr(&empty[buf]));
        }
        commit_to(smem_addr(&done));  // covers every MMA issued before it
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its 32 rows)
        if (!bar_wait(smem_addr(&done), 0u)) s_fail = 1;
        fence_after();
        // (FP32 sums of the accumulators and the power-of-two scaling, the widening to
        // FP64 with integer operations: GB300's FP64 pipe runs at 1/64 of the FP32 rate
        // and FP64 arithmetic here took longer than the whole MMA loop)
        const int q = warp & 3;
        const int64_t row = (int64_t)tile * T16_M + 32 * q + lane;
        const int nread = S < nacc ? S : nacc;
        const float sa = ldexpf(1.0f, -br.eA);
        for (int c0 = 0; c0 < P.RP && !s_fail; c0 += 8) {
            float re[8] = {0, 0, 0, 0, 0, 0, 0, 0}, im[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int acc = 0; acc < nread; ++acc) {
                uint32_t v[8], w[8];
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * nb + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n\t"
                    "tcgen05.wait::ld.sync.aligned;"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                    : "r"(ta), "r"(ta + (uint32_t)P.RP)
                    : "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    re[j] += __uint_as_float(v[j]);
                    im[j] += __uint_as_float(w[j]);
                }
            }
            if (row < br.N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int r = c0 + j;
                    if (r >= P.R) continue;
                    const float sb = ldexpf(1.0f, -P.eB[b * P.RP + r]);
                    const double zr = widen(re[j] * sa * sb), zi = widen(im[j] * sa * sb);
                    double* zz = z + 2 * ((int64_t)r * P.n + br.base + row);
                    if (gridDim.y == 1) {
                        zz[0] = zr;
                        zz[1] = zi;
                    } else {  // K ranges of other CTAs add into a zeroed z
                        atomicAdd(zz, zr);
                        atomicAdd(zz + 1, zi);
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) atomicOr(err, 1);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

int64_t padded_k(int64_t N) { return (4 * N + T16_KS - 1) / T16_KS * T16_KS; }

}  // namespace

bem_status tc16_build(const float2* const a1[4], const float2* const a2[4], const int64_t N[4], Tc16Ops& out,
                      cudaStream_t s, bool bf16) {
    out.bf16 = bf16;
    DevBuf mx;
    BEM_TRY(mx.alloc(4 * sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(mx.p, 0, 4 * sizeof(int), s));
    for (int b = 0; b < 4; ++b) {
        const int64_t cnt = 2 * N[b] * N[b];
        if (cnt == 0) continue;  // an empty block row (single-trace systems use two)
        BEM_LAUNCH(k_t16_absmax, 152 * 4, 256, 0, s, reinterpret_cast<const float*>(a1[b]), cnt, mx.as<int>() + b);
        BEM_LAUNCH(k_t16_absmax, 152 * 4, 256, 0, s, reinterpret_cast<const float*>(a2[b]), cnt, mx.as<int>() + b);
    }
    int hm[4];
    BEM_CUDA_TRY(cudaMemcpyAsync(hm, mx.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int b = 0; b < 4; ++b) {
        float m;
        std::memcpy(&m, &hm[b], sizeof(m));
        out.N[b] = N[b];
        out.Kp[b] = padded_k(N[b]);
        out.eA[b] = top_exponent(m);
        if (N[b] == 0) continue;
        // whole row tiles (the rows past N and the K padding stay zero)
        const size_t bytes = (size_t)((N[b] + T16_M - 1) / T16_M * T16_M) * out.Kp[b] * 2;
        BEM_TRY(out.hi[b].alloc(bytes, s));
        BEM_TRY(out.lo[b].alloc(bytes, s));
        BEM_CUDA_TRY(cudaMemsetAsync(out.hi[b].p, 0, bytes, s));
        BEM_CUDA_TRY(cudaMemsetAsync(out.lo[b].p, 0, bytes, s));
        if (out.bf16)
            BEM_LAUNCH(k_t16_split_ops<BF16>, 152 * 8, 256, 0, s, reinterpret_cast<const float*>(a1[b]),
                       reinterpret_cast<const float*>(a2[b]), N[b], out.Kp[b], ldexpf(1.0f, out.eA[b]),
                       out.hi[b].as<__half>(), out.lo[b].as<__half>());
        else
            BEM_LAUNCH(k_t16_split_ops<F16>, 152 * 8, 256, 0, s, reinterpret_cast<const float*>(a1[b]),
                       reinterpret_cast<const float*>(a2[b]), N[b], out.Kp[b], ldexpf(1.0f, out.eA[b]),
                       out.hi[b].as<__half>(), out.lo[b].as<__half>());
    }
    return BEM_OK;
}

size_t tc16_workspace_bytes(const int64_t N[4], int RP) {
    size_t total = 4 * 128 * sizeof(int) + 4 * 128 * sizeof(int);  // column maxima and exponents
    for (int b = 0; b < 4; ++b) total += 2 * (size_t)(2 * RP) * padded_k(N[b]) * 2;
    return total;
}

bem_status mtf_product_tc16(const Tc16Ops& ops, const double c1[4], const double c2[4], const int64_t base[4],
                            const int64_t x1[4], const int64_t x2[4], int64_t n, int R, const double2* x,
                            double2* z, void* work, size_t work_bytes, int* err, cudaStream_t s) {
    const int RP = tc_padded_columns(R);
    if (R < 1 || 2 * RP > 256) {
        set_error("FP16 tensor-core product: 1 to 128 right-hand sides per call");
        return BEM_E_INVALID_ARG;
    }
    if (work_bytes < tc16_workspace_bytes(ops.N, RP)) {
        set_error("FP16 tensor-core product: workspace too small");
        return BEM_E_INTERNAL;
    }
    char* w = static_cast<char*>(work);
    int* xmax = reinterpret_cast<int*>(w);
    int* eB = xmax + 4 * 128;
    w += 2 * 4 * 128 * sizeof(int);
    T16Prep pp{};
    T16Args A{};  // kernel parameters (copied at launch)
    int tiles = 0, min_stages = 1 << 30;
    for (int b = 0; b < 4; ++b) {
        const size_t bytes = (size_t)(2 * RP) * ops.Kp[b] * 2;
        pp.bh[b] = reinterpret_cast<__half*>(w);
        pp.bl[b] = reinterpret_cast<__half*>(w + bytes);
        w += 2 * bytes;
        pp.N[b] = ops.N[b];
        pp.Kp[b] = ops.Kp[b];
        pp.x1[b] = x1[b];
        pp.x2[b] = x2[b];
        pp.c1[b] = c1[b];
        pp.c2[b] = c2[b];
        T16Row& br = A.br[b];
        if (ops.N[b] == 0) continue;  // no tiles: the kernel never reads this block row
        A.ah[b] = ops.hi[b].as<__half>();
        A.al[b] = ops.lo[b].as<__half>();
        A.bh[b] = pp.bh[b];
        A.bl[b] = pp.bl[b];
        br.N = ops.N[b];
        br.base = base[b];
        br.stages = (int)(ops.Kp[b] / T16_KS);
        br.tiles = (int)((ops.N[b] + T16_M - 1) / T16_M);
        br.eA = ops.eA[b];
        tiles += br.tiles;
        min_stages = std::min(min_stages, br.stages);
    }
    // B rows past R and the K padding must read as zeros (A's padding is zero, and a
    // non-finite B entry there would reach every row)
    const size_t bbytes = (size_t)(w - reinterpret_cast<char*>(work)) - 2 * 4 * 128 * sizeof(int);
    if (bbytes) BEM_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(work) + 2 * 4 * 128 * sizeof(int), 0, bbytes, s));
    if (tiles == 0) return BEM_OK;
    pp.R = R;
    pp.RP = RP;
    pp.n = n;
    A.eB = eB;
    A.R = R;
    A.RP = RP;
    A.n = n;
    BEM_CUDA_TRY(cudaMemsetAsync(xmax, 0, 128 * sizeof(int), s));
    BEM_LAUNCH(k_t16_colmax, dim3(64, R), 256, 0, s, x, n, R, xmax);
    BEM_LAUNCH(k_t16_scales, 4, 128, 0, s, pp, xmax, eB);
    int64_t nmax = 0;
    for (int b = 0; b < 4; ++b) nmax = std::max(nmax, ops.N[b]);
    const dim3 pgrid((unsigned)std::min<int64_t>(64, (2 * nmax + 255) / 256), R, 4);
    if (ops.bf16) BEM_LAUNCH(k_t16_prep<BF16>, pgrid, 256, 0, s, pp, x, eB);
    else BEM_LAUNCH(k_t16_prep<F16>, pgrid, 256, 0, s, pp, x, eB);
    // K split: the wave efficiency of tiles * ksplit CTAs (one per SM) over 1..8
    int sms = 0, dev = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int ksplit = 1;
    double best = 0.0;
    for (int k = 1; k <= std::min(8, min_stages); ++k) {
        const int64_t ctas = (int64_t)tiles * k;
        const double eff = (double)ctas / (double)(sms * ((ctas + sms - 1) / sms));
        if (eff > best + 0.02) {
            best = eff;
            ksplit = k;
        }
    }
    A.ksplit = ksplit;
    const int nb = 2 * RP;
    const int stage_bytes = 2 * T16_A_PART + 2 * nb * T16_KS * 2;
    const int NS = stage_bytes <= 48 * 1024 ? 4 : stage_bytes <= 64 * 1024 ? 3 : 2;
    const int smem = NS * stage_bytes + 1024;
    if (ksplit > 1) BEM_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)R * n * sizeof(double2), s));
    if (ops.bf16) {
        BEM_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc16<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        BEM_LAUNCH(k_gemm_tc16<BF16>, dim3(tiles, ksplit), T16_THREADS, smem, s, A, reinterpret_cast<double*>(z),
                   err);
    } else {
        BEM_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc16<F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        BEM_LAUNCH(k_gemm_tc16<F16>, dim3(tiles, ksplit), T16_THREADS, smem, s, A, reinterpret_cast<double*>(z),
                   err);
    }
    return BEM_OK;
}

}  // namespace bem
