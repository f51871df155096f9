// Dense operator products on the tiled, symmetry-packed storage (the a9 step of the
// solve: the dense blocks of eq. mtf:discrete and of the other formulations applied to
// Krylov vectors, Sec. 3.3 / Sec. 5.1).
//
// Storage (bem_internal.cuh): per grid K as all 64 x 64 tiles, V and D as the tiles of
// the upper tile triangle (V, D are complex symmetric; Sec. 2.1 with Galerkin P1), and
// no T: T = K^T (Sec. 2.1).  One set of a product computes
//     y1 = cK K xa + cV V xb,     y2 = cD D xc + cT K^T xd,
// which covers the Calderon blocks of every formulation, reading each stored tile once:
// a tile A contributes its row sums A x (to the rows of its tile row) and, for K and
// for the off-diagonal tiles of V and D, its column sums A^T y (to the rows of its tile
// column).  Bytes per product: 3 N^2 entries per grid instead of the 4 N^2 of four full
// blocks (2 N^2 + N^2 for V, D, K).
//
// Work item = a tile pair (I, J), I <= J, of one set: the tiles K_IJ, K_JI, V_IJ, D_IJ
// (K_II, V_II, D_II on the diagonal), four tiles with the same four output slices
// y1[I], y1[J], y2[I], y2[J].  Persistent CTAs take items round-robin.  In each CTA one
// producer thread streams the item's tiles into a ring of 32 KB shared-memory stages with
// cp.async.bulk (one bulk copy per stage: a complex64 tile, or half a complex128 tile),
// completing on the stage's mbarrier; eight consumer warps compute from shared memory and
// release the stage through a second mbarrier.  Row sums: lanes own two columns, the 32
// lane partials of a group of rows are reduced by a butterfly that leaves one (row,
// column, re/im) value per lane pair; column sums: lanes accumulate their two columns over
// the warp's rows, then the eight warps' partials are added in shared memory.  An item's
// four output slices go to a partial-sum buffer (one slot per (output tile row, item
// column)), and a second kernel adds the slots of each output row in a fixed order, so
// the product is deterministic.
//
// Arithmetic: TP_F32 (complex64 matrices and x, FP32 products, ~1e-7: the inner products
// of the mixed mode); TP_DD (double-float on the FP32 pipe: x as FP32 high + low parts,
// complex128 entries split into high + low parts with integer operations, exact
// two-products and two-sums; the stored operator applied to ~1e-14 without the FP64
// pipe, which on this part is 1/64 of the FP32 pipe).
//
// Every mbarrier wait is bounded (TP_WAIT_LIMIT polls); a wait that gives up sets the
// error flag and makes the CTA skip the rest of its work (all consumer warps follow the
// same control flow, so no named barrier is left waiting); the producer waits, bounded,
// for the copies it issued before it returns.
#include "bem_internal.cuh"

#include <algorithm>
#include <cmath>

namespace bem {

namespace {

constexpr int TP_CHUNK = 32768;                   // bytes per ring stage (one bulk copy)
constexpr int TP_SMEM_LIMIT = 232448;             // 227 KB of shared memory per CTA
constexpr long long TP_WAIT_LIMIT = 1ll << 27;    // mbarrier polls before giving up (about a second)

__device__ __forceinline__ uint32_t s_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mb_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mb_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mb_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(bar)) : "memory");
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mb_wait(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < TP_WAIT_LIMIT; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(s_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// one bulk copy global -> shared completing on bar (16-byte aligned, size multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s_addr(dst)),
                 "l"(src), "r"(bytes), "r"(s_addr(bar))
                 : "memory");
}

// barrier of the consumer warps only (the producer warp never joins)
template <int W>
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * W) : "memory"); }

// ---- double-float arithmetic (error-free transformations on the FP32 pipe) ----
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (h, l) += (bh, bl); symmetric in its two operands (the same bits for a + b and b + a),
// so that a butterfly gives the same sums whichever lane keeps which half
__device__ __forceinline__ void dd_add(float& h, float& l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    h = s;
    l = __fadd_rn(__fadd_rn(l, bl), e);
}
// (h, l) += a (ah + al) times x (xh + xl): the main product exactly (two-product by FMA),
// the cross terms rounded (2^-24 of the main term), al xl dropped (2^-48)
template <bool AL>
__device__ __forceinline__ void dd_mac(float& h, float& l, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    float e = fmaf(ah, xh, -p);
    e = fmaf(ah, xl, e);
    if (AL) e = fmaf(al, xh, e);
    float s, t;
    two_sum(h, p, s, t);
    h = s;
    l = __fadd_rn(l, __fadd_rn(t, e));
}

// a double split into FP32 high and low parts with integer operations only (no FP64
// conversion instructions): hi = the leading 24 significand bits (truncated), lo = the
// next 29 rounded to FP32; |a - hi - lo| <= 2^-48 |a|.  Magnitudes below 2^-100 give 0.
__device__ __forceinline__ void split_double(double a, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF) - 1023;  // unbiased exponent
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e < -100 || e > 127) {  // zero, tiny, or outside the FP32 range (not reached by operator entries)
        hi = 0.0f;
        lo = 0.0f;
        return;
    }
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
    // the remaining 29 bits hold rest * 2^(e - 52) = (rest * 2^-29) * 2^(e - 23): the integer
    // rounded to FP32, then two exact power-of-two scalings (2^(e - 23) is a normal FP32
    // number for -100 <= e <= 127)
    const unsigned rest = (unsigned)(m & 0x1FFFFFFFull);
    const float r = __uint2float_rn(rest) * 1.8626451492309570e-9f;  // 2^-29
    const float sc = __uint_as_float((unsigned)(e - 23 + 127) << 23);
    lo = __uint_as_float(__float_as_uint(r * sc) | sign);
}

template <class ST>
struct Store;
template <>
struct Store<float2> {  // complex64 tile: 64 rows of 512 bytes, one chunk
    static constexpr int RPC = 64;
    static constexpr int CHUNKS = 1;
    static constexpr bool AL = false;
    // lane's columns: 2l, 2l+1 (one 16-byte load)
    __device__ static int col(int lane, int k) { return 2 * lane + k; }
    __device__ static void load(const unsigned char* row, int lane, float ah[4], float al[4]) {
        const float4 v = *reinterpret_cast<const float4*>(row + 16 * lane);
        ah[0] = v.x; ah[1] = v.y; ah[2] = v.z; ah[3] = v.w;
        al[0] = al[1] = al[2] = al[3] = 0.0f;
    }
    static constexpr int ROW_BYTES = 512;
};
template <>
struct Store<double2> {  // complex128 tile: 64 rows of 1024 bytes, two chunks of 32 rows
    static constexpr int RPC = 32;
    static constexpr int CHUNKS = 2;
    static constexpr bool AL = true;
    // lane's columns: l and l + 32 (two contiguous 512-byte warp loads)
    __device__ static int col(int lane, int k) { return lane + 32 * k; }
    __device__ static void load(const unsigned char* row, int lane, float ah[4], float al[4]) {
        const double2 u = *reinterpret_cast<const double2*>(row + 16 * lane);
        const double2 v = *reinterpret_cast<const double2*>(row + 512 + 16 * lane);
        split_double(u.x, ah[0], al[0]);
        split_double(u.y, ah[1], al[1]);
        split_double(v.x, ah[2], al[2]);
        split_double(v.y, ah[3], al[3]);
    }
    static constexpr int ROW_BYTES = 1024;
};

// x element / accumulator element per arithmetic
template <int MODE>
struct Arith;
template <>
struct Arith<TP_F32> {
    using X = float2;  // complex64 input
    using A = float2;  // accumulator (re, im)
    static constexpr int VAL = 1;  // floats per real value
};
template <>
struct Arith<TP_DD> {
    using X = float4;  // (re hi, im hi, re lo, im lo)
    using A = float4;  // same layout
    static constexpr int VAL = 2;
};

// Launch shape per (storage, arithmetic, columns).  Consumer warps W: 16 for one
// column, 8 for more (registers).  Half of them are row warps: one lane per tile row,
// the 64 columns split into W/4 blocks; the other half column warps: one lane per tile
// column, the 64 rows split into W/4 blocks.  Neither needs a cross-lane reduction; the
// W/4 block partials of each output are added once per item.
template <class ST, int MODE, int R>
struct Cfg {
    using X = typename Arith<MODE>::X;
    using A = typename Arith<MODE>::A;
    static constexpr int W = R == 1 ? 16 : 8;
    static constexpr int THREADS = 32 * (W + 1);
    static constexpr int NB = W / 4;      // blocks per half (column blocks of row warps, row blocks of column warps)
    static constexpr int BW = 64 / NB;    // block width (columns) or height (rows)
    static constexpr int CH = Store<ST>::CHUNKS;
    static constexpr int XSN = 8 * R * 64;  // elements of one set of input slices
    // input-slice elements per consumer thread; the next item's are prefetched into
    // registers while the current item streams when there are at most two (then the
    // slices are double-buffered by item)
    static constexpr int XPT = (XSN + 32 * W - 1) / (32 * W);
    static constexpr bool PREFETCH = XPT <= 2;
    static constexpr int NBUF = PREFETCH ? 2 : 1;
    static constexpr int XS = NBUF * XSN * (int)sizeof(X);
    static constexpr int RED = W * 3 * R * 32 * (int)sizeof(A);  // per-warp partials of three slots
    static constexpr int FIXED = XS + RED + 1024;
    static constexpr int S0 = (TP_SMEM_LIMIT - FIXED) / TP_CHUNK;
    static constexpr int S = S0 > 6 ? 6 : S0;  // ring stages
    static constexpr int BYTES = S * TP_CHUNK + FIXED;
    static constexpr int EMPTY = W / CH;  // warps reading each chunk
    static_assert(S >= 2, "shared-memory budget");
};

struct TileLaunch {
    const TileSet* sets;
    const int2* items;  // (set, I << 16 | J)
    int rc;             // columns of x and z (<= R)
    int64_t nitems;
    int64_t n;          // column length of x and z
    const void* x;
    void* part;
    int* err;
};

// The item's tiles in their fixed order: 0 = K_IJ, 1 = K_JI (I < J), 2 = V_IJ, 3 = D_IJ.
// Returns the count; src[] their first bytes.
template <class ST>
__device__ __forceinline__ int item_tiles(const TileSet& S, int I, int J, const unsigned char* src[4]) {
    const int f = S.flags;
    const int64_t nt = S.nt;
    const size_t tb = (size_t)OPT * OPT * sizeof(ST);
    int m = 0;
    if (f & (TS_KROW | TS_KCOL)) {
        src[m++] = static_cast<const unsigned char*>(S.K) + (size_t)(I * nt + J) * tb;
        if (I != J) src[m++] = static_cast<const unsigned char*>(S.K) + (size_t)(J * nt + I) * tb;
    }
    if (f & TS_V) src[m++] = static_cast<const unsigned char*>(S.V) + (size_t)op_sym_tile(I, J, nt) * tb;
    if (f & TS_D) src[m++] = static_cast<const unsigned char*>(S.D) + (size_t)op_sym_tile(I, J, nt) * tb;
    return m;
}

// exact product a x of an entry a = ah + al and an input x = xh + xl: p + e (p = fl(ah xh),
// e its exact error plus the rounded cross terms)
template <bool AL>
__device__ __forceinline__ void dd_prod(float ah, float al, float xh, float xl, float& p, float& e) {
    p = __fmul_rn(ah, xh);
    e = fmaf(ah, xh, -p);
    e = fmaf(ah, xl, e);
    if (AL) e = fmaf(al, xh, e);
}

// accumulators (re, im) += a (ar, ai) times x, in the product's arithmetic: FP32, or
// double-float (two exact products per part, one two-sum, one double-float add)
template <int MODE, bool AL>
__device__ __forceinline__ void cmac(float (&acc)[2][MODE == TP_DD ? 2 : 1], float arh, float aih, float arl,
                                     float ail, const typename Arith<MODE>::X& x) {
    if constexpr (MODE == TP_F32) {
        acc[0][0] = fmaf(arh, x.x, fmaf(-aih, x.y, acc[0][0]));
        acc[1][0] = fmaf(arh, x.y, fmaf(aih, x.x, acc[1][0]));
    } else {
        float p0, e0, p1, e1, s_, t_;
        dd_prod<AL>(arh, arl, x.x, x.z, p0, e0);
        dd_prod<AL>(-aih, -ail, x.y, x.w, p1, e1);
        two_sum(p0, p1, s_, t_);
        dd_add(acc[0][0], acc[0][1], s_, __fadd_rn(__fadd_rn(e0, e1), t_));
        dd_prod<AL>(arh, arl, x.y, x.w, p0, e0);
        dd_prod<AL>(aih, ail, x.x, x.z, p1, e1);
        two_sum(p0, p1, s_, t_);
        dd_add(acc[1][0], acc[1][1], s_, __fadd_rn(__fadd_rn(e0, e1), t_));
    }
}

// one stored entry (complex64 exact, or complex128 split into high + low parts)
template <class ST>
__device__ __forceinline__ void entry_at(const unsigned char* p, float& arh, float& aih, float& arl, float& ail) {
    if constexpr (sizeof(ST) == 8) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        arh = v.x; aih = v.y; arl = 0.f; ail = 0.f;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        split_double(v.x, arh, arl);
        split_double(v.y, aih, ail);
    }
}

// Per-warp role in a tile (see Cfg): row warp (rows 32 half + lane, columns of block
// blk) or column warp (column 32 half + lane, rows of block blk)
template <class ST, int MODE, int R>
struct Role {
    bool row;
    int half, blk, chunk;  // chunk: which 32 KB chunk of a complex128 tile the warp reads
};

// the tile's work of one warp: ROW: row sums of its lane's row over its column block into
// register slot RS; else column sums of its lane's column over its row block into slot CS
template <class ST, int MODE, int R, bool ROW>
__device__ __forceinline__ void tile_warp(const unsigned char* chunk, int half, int blk, int lane,
                                          const typename Arith<MODE>::X* __restrict__ xsl,
                                          float (&acc)[R][2][MODE == TP_DD ? 2 : 1]) {
    using C = Cfg<ST, MODE, R>;
    using X = typename Arith<MODE>::X;
    constexpr int RB = Store<ST>::ROW_BYTES;
    constexpr int RPC = Store<ST>::RPC;
    constexpr bool AL = Store<ST>::AL;
    if constexpr (ROW) {
        // lane's row in the chunk; its column block in 16-byte pieces visited from a
        // lane-dependent start, so that the 32 lanes' loads fall in distinct bank groups
        const int lrow = C::CH == 1 ? 32 * half + lane : lane;
        constexpr int EP = 16 / (int)sizeof(ST);  // entries per 16-byte piece
        constexpr int NP = C::BW / EP;            // pieces per block row
        const unsigned char* rp = chunk + (size_t)lrow * RB + (size_t)blk * C::BW * sizeof(ST);
#pragma unroll 4
        for (int c = 0; c < NP; ++c) {
            const int k = (c + lane) & (NP - 1);
            const int col = blk * C::BW + k * EP;
#pragma unroll
            for (int e = 0; e < EP; ++e) {
                float arh, aih, arl, ail;
                entry_at<ST>(rp + (k * EP + e) * sizeof(ST), arh, aih, arl, ail);
#pragma unroll
                for (int r = 0; r < R; ++r) cmac<MODE, AL>(acc[r], arh, aih, arl, ail, xsl[r * 64 + col + e]);
            }
        }
    } else {
        const int col = 32 * half + lane;
        const int row0 = blk * C::BW;
        const int lrow0 = C::CH == 1 ? row0 : row0 - RPC * (row0 / RPC);
#pragma unroll 4
        for (int t = 0; t < C::BW; ++t) {
            float arh, aih, arl, ail;
            entry_at<ST>(chunk + (size_t)(lrow0 + t) * RB + (size_t)col * sizeof(ST), arh, aih, arl, ail);
#pragma unroll
            for (int r = 0; r < R; ++r) cmac<MODE, AL>(acc[r], arh, aih, arl, ail, xsl[r * 64 + row0 + t]);
        }
    }
}

template <class ST, int MODE, int R>
__global__ void __launch_bounds__(Cfg<ST, MODE, R>::THREADS, 1) k_tile(TileLaunch L) {
    using C = Cfg<ST, MODE, R>;
    using X = typename C::X;
    using A = typename C::A;
    constexpr int W = C::W, S = C::S, CH = C::CH;
    constexpr int VAL = Arith<MODE>::VAL;
    constexpr int NT = 32 * W;  // consumer threads
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* stages = sm;
    X* xs0 = reinterpret_cast<X*>(sm + S * TP_CHUNK);                 // [NBUF][8][R][64]
    A* red = reinterpret_cast<A*>(sm + S * TP_CHUNK + C::XS);         // [W][3][R][32]
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + S * TP_CHUNK + C::XS + C::RED);
    uint64_t* empty = full + S;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mb_init(&full[i], 1);
            mb_init(&empty[i], C::EMPTY);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == W) {  // ---------------------------------------------------- producer
        if (lane == 0) {
            uint32_t q = 0;
            bool ok = true;
            for (int64_t k = blockIdx.x; k < L.nitems && ok; k += gridDim.x) {
                const int2 it = L.items[k];
                const unsigned char* src[4];
                const int ntl = item_tiles<ST>(L.sets[it.x], it.y >> 16, it.y & 0xFFFF, src);
                for (int t = 0; t < ntl && ok; ++t)
                    for (int h = 0; h < CH && ok; ++h, ++q) {
                        const int st = (int)(q % S);
                        if (q >= (uint32_t)S && !mb_wait(&empty[st], ((q / S) - 1) & 1)) {
                            ok = false;
                            break;
                        }
                        if (*abort_flag) {
                            ok = false;
                            break;
                        }
                        mb_expect_tx(&full[st], TP_CHUNK);
                        bulk_load(stages + (size_t)st * TP_CHUNK, src[t] + (size_t)h * TP_CHUNK, TP_CHUNK, &full[st]);
                    }
            }
            if (!ok) {
                atomicOr(L.err, 4);
                *abort_flag = 1;
            }
            // the copies issued last must land before the CTA may exit
            const uint32_t first = q > (uint32_t)S ? q - S : 0;
            for (uint32_t j = first; j < q; ++j) mb_wait(&full[j % S], (j / S) & 1);
        }
        return;
    }

    // ------------------------------------------------------------------ consumers
    const bool roww = warp < W / 2;
    const int ww = roww ? warp : warp - W / 2;
    const int half = ww & 1, blk = ww >> 1;
    // the chunk of a two-chunk (complex128) tile this warp reads: rows 32 half.. (row
    // warps) or the rows of its block (column warps)
    const int mychunk = CH == 1 ? 0 : (roww ? half : (blk * C::BW) / Store<ST>::RPC);
    const X* __restrict__ xg = static_cast<const X*>(L.x);
    // scaled input element e (slice, column, entry) of item (set St, tiles I, J)
    auto load_x = [&](const TileSet& St, int I, int J, int e) -> X {
        const int sl = e / (R * 64), r = (e / 64) % R, j = e % 64;
        const int tile = (sl == 0 || sl == 2 || sl == 4 || sl == 7) ? J : I;
        const int ci = sl >> 1;
        const int64_t off = ci == 0 ? St.xa : ci == 1 ? St.xb : ci == 2 ? St.xc : St.xd;
        const int64_t row = (int64_t)tile * 64 + j;
        const float ch = St.ch[ci], cl = St.cl[ci];
        X v{};
        if (r < L.rc && row < St.N && (ch != 0.0f || cl != 0.0f)) {
            const X u = xg[(int64_t)r * L.n + off + row];
            if constexpr (MODE == TP_F32) {
                v = make_float2(ch * u.x, ch * u.y);
            } else {
                // (u.hi + u.lo) (ch + cl) as a double-float pair per component
                float pr = __fmul_rn(u.x, ch), pi = __fmul_rn(u.y, ch);
                float er = fmaf(u.x, ch, -pr), ei = fmaf(u.y, ch, -pi);
                er = fmaf(u.x, cl, fmaf(u.z, ch, er));
                ei = fmaf(u.y, cl, fmaf(u.w, ch, ei));
                float sr, tr, si, ti;
                two_sum(pr, er, sr, tr);
                two_sum(pi, ei, si, ti);
                v = make_float4(sr, si, tr, ti);
            }
        }
        return v;
    };
    X pre[C::PREFETCH ? C::XPT : 1];
    if constexpr (C::PREFETCH) {
        if (blockIdx.x < L.nitems) {
            const int2 it = L.items[blockIdx.x];
            const TileSet& St = L.sets[it.x];
#pragma unroll
            for (int u = 0; u < C::XPT; ++u) {
                const int e = threadIdx.x + u * NT;
                pre[u] = e < C::XSN ? load_x(St, it.y >> 16, it.y & 0xFFFF, e) : X{};
            }
        }
    }
    uint32_t q = 0;
    bool aborted = false;
    int par = 0;
    for (int64_t k = blockIdx.x; k < L.nitems; k += gridDim.x, par ^= 1) {
        const int2 it = L.items[k];
        const TileSet& St = L.sets[it.x];
        const int I = it.y >> 16, J = it.y & 0xFFFF;
        const bool diag = I == J;
        const int flags = St.flags;
        X* xs = xs0 + (C::NBUF == 2 ? par : 0) * C::XSN;
        // item start: this item's scaled input slices (the previous item's readers of this
        // buffer passed the end-of-item barrier before any thread got here)
        if constexpr (C::PREFETCH) {
#pragma unroll
            for (int u = 0; u < C::XPT; ++u) {
                const int e = threadIdx.x + u * NT;
                if (e < C::XSN) xs[e] = pre[u];
            }
            const int64_t kn = k + gridDim.x;  // the next item's inputs, in flight meanwhile
            if (kn < L.nitems) {
                const int2 itn = L.items[kn];
                const TileSet& Sn = L.sets[itn.x];
#pragma unroll
                for (int u = 0; u < C::XPT; ++u) {
                    const int e = threadIdx.x + u * NT;
                    pre[u] = e < C::XSN ? load_x(Sn, itn.y >> 16, itn.y & 0xFFFF, e) : X{};
                }
            }
        } else {
            for (int e = threadIdx.x; e < C::XSN; e += NT) xs[e] = load_x(St, I, J, e);
        }
        consumers_sync<W>();
        // per-lane partials: row warps slots 0, 1, 2 (y1_I, y1_J, y2_I), column warps
        // slots 1, 2, 3 (y1_J, y2_I, y2_J), R columns, (re, im), double-float pairs in TP_DD
        float acc[3][R][2][VAL];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int v = 0; v < VAL; ++v) acc[a][r][m][v] = 0.0f;
        // one tile: wait for the warp's chunk, compute, release it.  Kinds: K_IJ (row slot 0
        // from x_a(J); column slot y2_J = 3, or y2_I = 2 on the diagonal, from x_d(I)),
        // K_JI (row slot 1 from x_a(I); column slot 2 from x_d(J)), V_IJ (row 0 from x_b(J);
        // column 1 from x_b(I), off the diagonal), D_IJ (row 2 from x_c(J); column 3 from
        // x_c(I), off the diagonal).  Input slices: 0 xa_J, 1 xa_I, 2 xb_J, 3 xb_I, 4 xc_J,
        // 5 xc_I, 6 xd_I, 7 xd_J.
        auto tile = [&](int xr, int xc, int rs, int cs, bool do_row, bool do_col) {
            const uint32_t qq = q + mychunk;
            const int st = (int)(qq % S);
            if (!aborted && *abort_flag) aborted = true;
            if (!aborted && !mb_wait(&full[st], (qq / S) & 1)) {
                aborted = true;
                if (lane == 0) atomicOr(L.err, 8);
                *abort_flag = 1;
            }
            const unsigned char* chunk = stages + (size_t)st * TP_CHUNK;
            if (roww && do_row) {
                const X* xsl = xs + xr * R * 64;
                if (rs == 0) tile_warp<ST, MODE, R, true>(chunk, half, blk, lane, xsl, acc[0]);
                else if (rs == 1) tile_warp<ST, MODE, R, true>(chunk, half, blk, lane, xsl, acc[1]);
                else tile_warp<ST, MODE, R, true>(chunk, half, blk, lane, xsl, acc[2]);
            }
            if (!roww && do_col) {
                const X* xsl = xs + xc * R * 64;
                if (cs == 1) tile_warp<ST, MODE, R, false>(chunk, half, blk, lane, xsl, acc[0]);
                else if (cs == 2) tile_warp<ST, MODE, R, false>(chunk, half, blk, lane, xsl, acc[1]);
                else tile_warp<ST, MODE, R, false>(chunk, half, blk, lane, xsl, acc[2]);
            }
            __syncwarp();
            if (lane == 0) mb_arrive(&empty[st]);
            q += CH;
        };
        if (flags & (TS_KROW | TS_KCOL)) {
            tile(0, 6, 0, diag ? 2 : 3, (flags & TS_KROW) != 0, (flags & TS_KCOL) != 0);
            if (!diag) tile(1, 7, 1, 2, (flags & TS_KROW) != 0, (flags & TS_KCOL) != 0);
        }
        if (flags & TS_V) tile(2, 3, 0, 1, true, !diag);
        if (flags & TS_D) tile(4, 5, 2, 3, true, !diag);
        // item end: the warps' partials, then per output the block partials of the row
        // warps and the column warps added in a fixed order, into the partial-sum slots
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                A v;
                if constexpr (MODE == TP_F32) v = make_float2(acc[a][r][0][0], acc[a][r][1][0]);
                else v = make_float4(acc[a][r][0][0], acc[a][r][1][0], acc[a][r][0][1], acc[a][r][1][1]);
                red[((warp * 3 + a) * R + r) * 32 + lane] = v;
            }
        consumers_sync<W>();
        const bool y1 = (flags & TS_Y1) != 0, y2 = (flags & TS_Y2) != 0;
        const int64_t nt = St.nt;
        if (!aborted) {
            for (int e = threadIdx.x; e < 4 * R * 64; e += NT) {
                const int slot = e / (R * 64), r = (e / 64) % R, o = e % 64;
                if (diag && (slot == 1 || slot == 3)) continue;
                if ((slot < 2 && !y1) || (slot >= 2 && !y2) || r >= L.rc) continue;
                const int h = o >> 5, l = o & 31;
                A sum{};
#pragma unroll
                for (int side = 0; side < 2; ++side) {  // row warps (slots 0..2), column warps (slots 1..3)
                    const int a = side == 0 ? slot : slot - 1;
                    if (a < 0 || a > 2) continue;
#pragma unroll
                    for (int b = 0; b < C::NB; ++b) {
                        const int w = side * (W / 2) + h + 2 * b;
                        const A v = red[((w * 3 + a) * R + r) * 32 + l];
                        if constexpr (MODE == TP_F32) {
                            sum.x = __fadd_rn(sum.x, v.x);
                            sum.y = __fadd_rn(sum.y, v.y);
                        } else {
                            dd_add(sum.x, sum.z, v.x, v.z);
                            dd_add(sum.y, sum.w, v.y, v.w);
                        }
                    }
                }
                const int out = slot >> 1;
                const int64_t trow = (slot & 1) ? J : I, tcol = (slot & 1) ? I : J;
                const int64_t idx = St.part * R + ((((out * nt + trow) * nt + tcol) * R + r) << 6) + o;
                static_cast<A*>(L.part)[idx] = sum;
            }
        }
    }
}

// z rows of every active output: the sum over the partial-sum slots of the row's tile
// row in double-float, one CTA per (set, output, tile row) and column; the 64 rows x 4
// groups of slots (slot J to group J mod 4, the groups then added in order) give the
// same summation order for any number of columns, so a batched column equals the same
// column computed alone.
constexpr int RED_GROUPS = 4;
template <int MODE, int R>
__global__ void __launch_bounds__(64 * RED_GROUPS) k_tile_reduce(const TileSet* __restrict__ sets, int nsets,
                                                                 int64_t rtiles, int64_t n,
                                                                 const void* __restrict__ part,
                                                                 double2* __restrict__ z) {
    using A = typename Arith<MODE>::A;
    __shared__ float4 sh[64 * RED_GROUPS];
    const int64_t b = blockIdx.x;
    const int r = blockIdx.y;
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sets[mid].rtile0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const TileSet& St = sets[lo];
    const int64_t nt = St.nt;
    const int out = (int)((b - St.rtile0) / nt);
    const int64_t I = (b - St.rtile0) % nt;
    const int64_t yoff = out == 0 ? St.y1 : St.y2;
    if (yoff < 0) return;
    const int t = threadIdx.x;
    const int row = t & 63, jg = t >> 6;
    float sr = 0.f, srl = 0.f, si = 0.f, sil = 0.f;
    const A* __restrict__ p = static_cast<const A*>(part) + St.part * R + (((out * nt + I) * nt) * R << 6);
    for (int64_t J = jg; J < nt; J += RED_GROUPS) {
        const A a = p[((J * R + r) << 6) + row];
        if constexpr (MODE == TP_F32) {
            dd_add(sr, srl, a.x, 0.0f);
            dd_add(si, sil, a.y, 0.0f);
        } else {
            dd_add(sr, srl, a.x, a.z);
            dd_add(si, sil, a.y, a.w);
        }
    }
    sh[t] = make_float4(sr, si, srl, sil);
    __syncthreads();
    if (jg != 0) return;
    for (int g = 1; g < RED_GROUPS; ++g) {
        const float4 o = sh[t + g * 64];
        dd_add(sr, srl, o.x, o.z);
        dd_add(si, sil, o.y, o.w);
    }
    const int64_t gi = I * 64 + row;
    if (gi < St.N) z[(int64_t)r * n + yoff + gi] = make_double2((double)sr + (double)srl, (double)si + (double)sil);
}

template <class ST>
__global__ void k_tiles_to_dense(const ST* __restrict__ src, int layout, int transpose, int64_t N, int nt,
                                 ST* __restrict__ dst) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    int64_t i = e / N, j = e % N;
    if (transpose) {
        const int64_t t = i;
        i = j;
        j = t;
    }
    int64_t idx = op_index(layout, N, nt, i, j);
    if (idx < 0) idx = op_index(layout, N, nt, j, i);
    dst[e] = src[idx];
}

template <class ST, int MODE, int R>
bem_status launch_tile(const TileProd& P, int rc, const void* x, double2* z, void* part, int* err, cudaStream_t s) {
    using C = Cfg<ST, MODE, R>;
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_tile<ST, MODE, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::BYTES));
    int dev = 0, sms = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TileLaunch L;
    L.sets = P.dsets.as<TileSet>();
    L.items = P.ditems.as<int2>();
    L.rc = rc;
    L.nitems = P.items;
    L.n = P.n;
    L.x = x;
    L.part = part;
    L.err = err;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(P.items, sms));
    static const char* names[2][2][4] = {
        {{"k_tile<c64,f32,1>", "k_tile<c64,f32,2>", "k_tile<c64,f32,4>", "k_tile<c64,f32,8>"},
         {"k_tile<c64,dd,1>", "k_tile<c64,dd,2>", "k_tile<c64,dd,4>", "k_tile<c64,dd,8>"}},
        {{"k_tile<c128,f32,1>", "k_tile<c128,f32,2>", "k_tile<c128,f32,4>", "k_tile<c128,f32,8>"},
         {"k_tile<c128,dd,1>", "k_tile<c128,dd,2>", "k_tile<c128,dd,4>", "k_tile<c128,dd,8>"}}};
    const int ri = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : 3;
    BEM_LAUNCH_PTR(names[sizeof(ST) == 16][MODE][ri], (k_tile<ST, MODE, R>), grid, C::THREADS, C::BYTES, s, L);
    static const char* rnames[2][4] = {
        {"k_tile_reduce<f32,1>", "k_tile_reduce<f32,2>", "k_tile_reduce<f32,4>", "k_tile_reduce<f32,8>"},
        {"k_tile_reduce<dd,1>", "k_tile_reduce<dd,2>", "k_tile_reduce<dd,4>", "k_tile_reduce<dd,8>"}};
    BEM_LAUNCH_PTR(rnames[MODE][ri], (k_tile_reduce<MODE, R>), dim3((unsigned)P.rtiles, (unsigned)rc),
                   64 * RED_GROUPS, 0, s, L.sets, (int)P.sets.size(), P.rtiles, P.n, part, z);
    return BEM_OK;
}

// ---- self-test helpers: seeded values and an FP64 dense reference -----------------
__device__ __forceinline__ double hash_unit(uint64_t i, uint64_t seed) {
    uint64_t h = i * 0x9E3779B97F4A7C15ull + seed;
    h ^= h >> 30;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    h *= 0x94D049BB133111EBull;
    h ^= h >> 31;
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);  // [0, 1), 53 bits
}

// complex entries with real parts in [0.5, 1) and imaginary parts in [-0.25, 0.25)
template <class T>
__global__ void k_fill_complex(T* __restrict__ a, int64_t count, uint64_t seed) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double re = 0.5 + 0.5 * hash_unit(2 * i, seed), im = -0.25 + 0.5 * hash_unit(2 * i + 1, seed);
    if constexpr (sizeof(T) == 8) a[i] = make_float2((float)re, (float)im);
    else a[i] = make_double2(re, im);
}

__global__ void k_round_c64(const double2* __restrict__ x, int64_t n, float2* __restrict__ y,
                            double2* __restrict__ xr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 f = make_float2((float)x[i].x, (float)x[i].y);
    y[i] = f;
    xr[i] = make_double2(f.x, f.y);
}

__global__ void k_split_dd(const double2* __restrict__ x, int64_t n, float4* __restrict__ xs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = x[i];
    const float hr = (float)v.x, hi = (float)v.y;
    xs[i] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
}

// y[i] += c sum_j A[i][j] x[j] in FP64, A dense row-major N x N (complex64 or complex128);
// one warp per row
template <class T>
__global__ void k_dense_ref(const T* __restrict__ A, int64_t N, const double2* __restrict__ x, double c,
                            double2* __restrict__ y) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    double sr = 0.0, si = 0.0;
    for (int64_t j = lane; j < N; j += 32) {
        const double ar = (double)A[i * N + j].x, ai = (double)A[i * N + j].y;
        sr += ar * x[j].x - ai * x[j].y;
        si += ar * x[j].y + ai * x[j].x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
        y[i].x += c * sr;
        y[i].y += c * si;
    }
}

}  // namespace

void tile_prod_add(TileProd& P, const void* K, const void* V, const void* D, int64_t N, double cK, double cV,
                   double cD, double cT, int64_t xa, int64_t xb, int64_t xc, int64_t xd, int64_t y1, int64_t y2) {
    TileSet t{};
    t.K = K;
    t.V = V;
    t.D = D;
    t.N = N;
    t.nt = op_tiles(N);
    const double c[4] = {K ? cK : 0.0, V ? cV : 0.0, D ? cD : 0.0, K ? cT : 0.0};
    for (int i = 0; i < 4; ++i) {
        t.c[i] = c[i];
        t.ch[i] = (float)c[i];
        t.cl[i] = (float)(c[i] - (double)t.ch[i]);
    }
    t.xa = xa; t.xb = xb; t.xc = xc; t.xd = xd;
    t.y1 = y1; t.y2 = y2;
    t.flags = (c[0] != 0.0 ? TS_KROW : 0) | (c[3] != 0.0 ? TS_KCOL : 0) | (c[1] != 0.0 ? TS_V : 0) |
              (c[2] != 0.0 ? TS_D : 0) | (y1 >= 0 ? TS_Y1 : 0) | (y2 >= 0 ? TS_Y2 : 0);
    t.item0 = P.items;
    t.rtile0 = P.rtiles;
    t.part = P.part_per_col;  // per column: the kernels place the set at part * R (R columns)
    P.items += (int64_t)t.nt * (t.nt + 1) / 2;
    P.rtiles += 2 * (int64_t)t.nt;
    P.part_per_col += 2 * (int64_t)t.nt * t.nt * OPT;
    P.sets.push_back(t);
}

bem_status tile_prod_finish(TileProd& P, int64_t n, int storage, cudaStream_t s) {
    BEM_REQUIRE(!P.sets.empty(), "a product without operators");
    BEM_REQUIRE(storage == 8 || storage == 16, "operator storage must be complex64 or complex128");
    P.n = n;
    P.storage = storage;
    std::vector<int2> items;
    items.reserve((size_t)P.items);
    for (size_t k = 0; k < P.sets.size(); ++k) {
        const int nt = P.sets[k].nt;
        BEM_REQUIRE(nt < 65536, "operator too large for the tile product (more than 4M vertices)");
        for (int I = 0; I < nt; ++I)
            for (int J = I; J < nt; ++J) items.push_back(make_int2((int)k, (I << 16) | J));
    }
    BEM_TRY(P.dsets.alloc(P.sets.size() * sizeof(TileSet), s));
    BEM_TRY(P.ditems.alloc(items.size() * sizeof(int2), s));
    BEM_CUDA_TRY(cudaMemcpyAsync(P.dsets.p, P.sets.data(), P.sets.size() * sizeof(TileSet), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(P.ditems.p, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    // the host vectors must outlive the copies
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    return BEM_OK;
}

size_t tile_part_bytes(const TileProd& P, int mode, int R) {
    const int Rt = R <= 1 ? 1 : R <= 2 ? 2 : R <= 4 ? 4 : 8;
    return (size_t)P.part_per_col * Rt * (mode == TP_F32 ? sizeof(float2) : sizeof(float4));
}

bem_status tile_product(const TileProd& P, int mode, int rc, const void* x, double2* z, void* part, int* err,
                        cudaStream_t s) {
    BEM_REQUIRE(rc >= 1 && rc <= 8, "tile products take 1 to 8 columns");
    BEM_REQUIRE(mode == TP_DD || P.storage == 8, "FP32 products need complex64 operators");
    if (mode == TP_DD && rc > 4) {  // double-float: at most 4 columns per launch (registers)
        BEM_TRY(tile_product(P, mode, 4, x, z, part, err, s));
        return tile_product(P, mode, rc - 4, static_cast<const float4*>(x) + 4 * P.n, z + 4 * P.n, part, err, s);
    }
    const int R = rc <= 1 ? 1 : rc <= 2 ? 2 : rc <= 4 ? 4 : 8;
    if (P.storage == 8) {
        if (mode == TP_F32) {
            switch (R) {
                case 1: return launch_tile<float2, TP_F32, 1>(P, rc, x, z, part, err, s);
                case 2: return launch_tile<float2, TP_F32, 2>(P, rc, x, z, part, err, s);
                case 4: return launch_tile<float2, TP_F32, 4>(P, rc, x, z, part, err, s);
                default: return launch_tile<float2, TP_F32, 8>(P, rc, x, z, part, err, s);
            }
        }
        switch (R) {
            case 1: return launch_tile<float2, TP_DD, 1>(P, rc, x, z, part, err, s);
            case 2: return launch_tile<float2, TP_DD, 2>(P, rc, x, z, part, err, s);
            default: return launch_tile<float2, TP_DD, 4>(P, rc, x, z, part, err, s);
        }
    }
    switch (R) {
        case 1: return launch_tile<double2, TP_DD, 1>(P, rc, x, z, part, err, s);
        case 2: return launch_tile<double2, TP_DD, 2>(P, rc, x, z, part, err, s);
        default: return launch_tile<double2, TP_DD, 4>(P, rc, x, z, part, err, s);
    }
}

bem_status tiles_to_dense(const void* src, int layout, bool transpose, int64_t N, int storage, void* dst,
                          cudaStream_t s) {
    const unsigned blocks = (unsigned)((N * N + 255) / 256);
    if (N == 0) return BEM_OK;
    if (storage == 8)
        BEM_LAUNCH(k_tiles_to_dense<float2>, blocks, 256, 0, s, static_cast<const float2*>(src), layout,
                   transpose ? 1 : 0, N, op_tiles(N), static_cast<float2*>(dst));
    else
        BEM_LAUNCH(k_tiles_to_dense<double2>, blocks, 256, 0, s, static_cast<const double2*>(src), layout,
                   transpose ? 1 : 0, N, op_tiles(N), static_cast<double2*>(dst));
    return BEM_OK;
}

}  // namespace bem

namespace bem {

bem_status random_tiled_ops(int64_t N, int storage, uint64_t seed, DevBuf tiles[3], DevBuf* dense, cudaStream_t s) {
    const int lay[3] = {OP_SYM, OP_FULL, OP_SYM};
    for (int m = 0; m < 3; ++m) {
        const int64_t cnt = (int64_t)op_entries(lay[m], N);
        BEM_TRY(tiles[m].alloc((size_t)cnt * storage, s));
        const unsigned b = (unsigned)((cnt + 255) / 256);
        if (storage == 8) BEM_LAUNCH(k_fill_complex<float2>, b, 256, 0, s, tiles[m].as<float2>(), cnt, seed + m);
        else BEM_LAUNCH(k_fill_complex<double2>, b, 256, 0, s, tiles[m].as<double2>(), cnt, seed + m);
    }
    if (!dense) return BEM_OK;
    for (int m = 0; m < 4; ++m) BEM_TRY(dense[m].alloc((size_t)N * N * storage, s));
    BEM_TRY(tiles_to_dense(tiles[0].p, OP_SYM, false, N, storage, dense[0].p, s));
    BEM_TRY(tiles_to_dense(tiles[1].p, OP_FULL, false, N, storage, dense[1].p, s));
    BEM_TRY(tiles_to_dense(tiles[1].p, OP_FULL, true, N, storage, dense[2].p, s));
    BEM_TRY(tiles_to_dense(tiles[2].p, OP_SYM, false, N, storage, dense[3].p, s));
    return BEM_OK;
}

// Two grids (300 and 170 vertices: ragged last tiles), the four operators of each as
// seeded random tiles, one set per grid with (cK, cV, cD, cT) = (-0.7, 1.3, 2.1, 0.4) and
// (-1, 1, 1, 1), R columns; the same product from dense copies of the tiles (T = the
// transposed copy of K) with an FP64 kernel.  Returns the relative L2 difference.
bem_status selftest_tile(int mode, int storage, int R, double* rel_err, cudaStream_t s) {
    BEM_REQUIRE(mode == TP_F32 || mode == TP_DD, "unknown arithmetic");
    BEM_REQUIRE(storage == 8 || storage == 16, "unknown storage");
    BEM_REQUIRE(mode == TP_DD || storage == 8, "FP32 products need complex64 operators");
    BEM_REQUIRE(R >= 1 && R <= 8, "1 to 8 columns");
    const int64_t Ns[2] = {300, 170};
    const int64_t n = 2 * Ns[0] + 2 * Ns[1];
    const double coef[2][4] = {{-0.7, 1.3, 2.1, 0.4}, {-1.0, 1.0, 1.0, 1.0}};
    DevBuf tiles[2][3], dense[2][4];  // [grid][V, K, D] and [grid][V, K, T, D]
    for (int g = 0; g < 2; ++g) BEM_TRY(random_tiled_ops(Ns[g], storage, 77 + 10 * g, tiles[g], dense[g], s));
    TileProd P;
    int64_t off = 0;
    for (int g = 0; g < 2; ++g) {
        const int64_t N = Ns[g];
        tile_prod_add(P, tiles[g][1].p, tiles[g][0].p, tiles[g][2].p, N, coef[g][0], coef[g][1], coef[g][2],
                      coef[g][3], off, off + N, off, off + N, off, off + N);
        off += 2 * N;
    }
    BEM_TRY(tile_prod_finish(P, n, storage, s));
    DevBuf x, xr, x32, xs, z, zr, part, err;
    BEM_TRY(x.alloc((size_t)R * n * 16, s));
    BEM_LAUNCH(k_fill_complex<double2>, (unsigned)((R * n + 255) / 256), 256, 0, s, x.as<double2>(), R * n, 999);
    BEM_TRY(xr.alloc((size_t)R * n * 16, s));
    BEM_TRY(x32.alloc((size_t)R * n * 8, s));
    BEM_TRY(xs.alloc((size_t)R * n * 16, s));
    BEM_TRY(z.alloc((size_t)R * n * 16, s));
    BEM_TRY(zr.alloc((size_t)R * n * 16, s));
    BEM_TRY(part.alloc(tile_part_bytes(P, mode, R), s));
    BEM_TRY(err.alloc(sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    BEM_CUDA_TRY(cudaMemsetAsync(z.p, 0, z.bytes, s));
    BEM_CUDA_TRY(cudaMemsetAsync(zr.p, 0, zr.bytes, s));
    const unsigned bx = (unsigned)((R * n + 255) / 256);
    if (mode == TP_F32) {  // the FP32 product sees x rounded to complex64: so does the reference
        BEM_LAUNCH(k_round_c64, bx, 256, 0, s, x.as<double2>(), R * n, x32.as<float2>(), xr.as<double2>());
        BEM_TRY(tile_product(P, TP_F32, R, x32.p, z.as<double2>(), part.p, err.as<int>(), s));
    } else {
        BEM_CUDA_TRY(cudaMemcpyAsync(xr.p, x.p, x.bytes, cudaMemcpyDeviceToDevice, s));
        BEM_LAUNCH(k_split_dd, bx, 256, 0, s, x.as<double2>(), R * n, xs.as<float4>());
        BEM_TRY(tile_product(P, TP_DD, R, xs.p, z.as<double2>(), part.p, err.as<int>(), s));
    }
    // reference: y1 = cK K xa + cV V xb, y2 = cD D xc + cT T xd per grid and column
    off = 0;
    for (int g = 0; g < 2; ++g) {
        const int64_t N = Ns[g];
        const unsigned br = (unsigned)((N * 32 + 255) / 256);
        for (int r = 0; r < R; ++r) {
            const double2* xv = xr.as<double2>() + (int64_t)r * n + off;
            double2* y1 = zr.as<double2>() + (int64_t)r * n + off;
            double2* y2 = y1 + N;
            // (matrix index in dense[g], input half, output, coefficient)
            const int mat[4] = {1, 0, 3, 2};
            const int in_half[4] = {0, 1, 0, 1};
            double2* outp[4] = {y1, y1, y2, y2};
            const double c[4] = {coef[g][0], coef[g][1], coef[g][2], coef[g][3]};
            for (int q = 0; q < 4; ++q) {
                if (storage == 8)
                    BEM_LAUNCH(k_dense_ref<float2>, br, 256, 0, s, dense[g][mat[q]].as<float2>(), N, xv + in_half[q] * N,
                               c[q], outp[q]);
                else
                    BEM_LAUNCH(k_dense_ref<double2>, br, 256, 0, s, dense[g][mat[q]].as<double2>(), N,
                               xv + in_half[q] * N, c[q], outp[q]);
            }
        }
        off += 2 * N;
    }
    std::vector<double2> h1((size_t)R * n), h2((size_t)R * n);
    int h_err = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(h1.data(), z.p, h1.size() * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(h2.data(), zr.p, h2.size() * 16, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err) {
        set_error("tile product: an mbarrier wait timed out");
        return BEM_E_INTERNAL;
    }
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < h1.size(); ++i) {
        const double dx = h1[i].x - h2[i].x, dy = h1[i].y - h2[i].y;
        num += dx * dx + dy * dy;
        den += h2[i].x * h2[i].x + h2[i].y * h2[i].y;
    }
    *rel_err = den > 0.0 ? std::sqrt(num / den) : 0.0;
    return BEM_OK;
}

}  // namespace bem
