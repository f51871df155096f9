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

constexpr int TP_WARPS = 8;                       // consumer warps
constexpr int TP_THREADS = 32 * (TP_WARPS + 1);   // + one producer warp
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

// barrier of the eight consumer warps only (the producer warp never joins)
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * TP_WARPS) : "memory"); }

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

// rows per butterfly group: at most 16 (row, column, re/im) values per lane
template <int R, int RPW>
struct Group {
    static constexpr int G = (8 / R) < RPW ? ((8 / R) < 1 ? 1 : 8 / R) : RPW;
    static constexpr int NV = G * R * 2;  // values per lane before the butterfly (<= 16)
};

template <class ST, int MODE, int R>
struct Layout {
    static constexpr int RPC = Store<ST>::RPC;
    static constexpr int RPW = RPC / TP_WARPS;  // rows per warp per chunk
    static constexpr int XS = 8 * R * 64 * (int)sizeof(typename Arith<MODE>::X);   // 8 input slices
    static constexpr int ACC = 4 * R * 64 * (int)sizeof(typename Arith<MODE>::A);  // 4 output slices
    static constexpr int RED = TP_WARPS * R * 64 * (int)sizeof(typename Arith<MODE>::A);
    static constexpr int FIXED = XS + ACC + RED + 1024;
    static constexpr int S0 = (TP_SMEM_LIMIT - FIXED) / TP_CHUNK;
    static constexpr int S = S0 > 6 ? 6 : S0;  // ring stages
    static constexpr int BYTES = S * TP_CHUNK + FIXED;
    static_assert(S >= 2, "shared-memory budget");
};

struct TileLaunch {
    const TileSet* sets;
    int nsets;
    int rc;         // columns of x and z (<= R)
    int64_t items;
    int64_t n;      // column length of x and z
    const void* x;
    void* part;
    int* err;
};

struct ItemInfo {
    int set, I, J;
};

__device__ ItemInfo decode_item(const TileSet* __restrict__ sets, int nsets, int64_t k) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sets[mid].item0 <= k) lo = mid;
        else hi = mid - 1;
    }
    const int64_t kk = k - sets[lo].item0;
    const int64_t nt = sets[lo].nt;
    // row I of the upper tile triangle starts at item I nt - I (I - 1) / 2
    const double b = 2.0 * (double)nt + 1.0;
    int64_t a = (int64_t)floor(0.5 * (b - sqrt(fmax(b * b - 8.0 * (double)kk, 0.0))));
    a = a < 0 ? 0 : (a > nt - 1 ? nt - 1 : a);
    while (a > 0 && op_sym_tile(a, a, nt) > kk) --a;
    while (a + 1 < nt && op_sym_tile(a + 1, a + 1, nt) <= kk) ++a;
    ItemInfo it;
    it.set = lo;
    it.I = (int)a;
    it.J = (int)(a + (kk - op_sym_tile(a, a, nt)));
    return it;
}

// The item's tiles in their fixed order: 0 = K_IJ, 1 = K_JI (I < J), 2 = V_IJ, 3 = D_IJ.
// Returns the count; kinds[] the tile kinds, src[] their first bytes.
template <class ST>
__device__ int item_tiles(const TileSet& S, int I, int J, int kinds[4], const unsigned char* src[4]) {
    const bool useK = S.K != nullptr && (S.c[0] != 0.0 || S.c[3] != 0.0);
    const bool useV = S.V != nullptr && S.c[1] != 0.0;
    const bool useD = S.D != nullptr && S.c[2] != 0.0;
    const int64_t nt = S.nt;
    const size_t tb = (size_t)OPT * OPT * sizeof(ST);
    int m = 0;
    if (useK) {
        kinds[m] = 0;
        src[m++] = static_cast<const unsigned char*>(S.K) + (size_t)(I * nt + J) * tb;
        if (I != J) {
            kinds[m] = 1;
            src[m++] = static_cast<const unsigned char*>(S.K) + (size_t)(J * nt + I) * tb;
        }
    }
    if (useV) {
        kinds[m] = 2;
        src[m++] = static_cast<const unsigned char*>(S.V) + (size_t)op_sym_tile(I, J, nt) * tb;
    }
    if (useD) {
        kinds[m] = 3;
        src[m++] = static_cast<const unsigned char*>(S.D) + (size_t)op_sym_tile(I, J, nt) * tb;
    }
    return m;
}

// Input slices of an item: 0 xa_J, 1 xa_I, 2 xb_J, 3 xb_I, 4 xc_J, 5 xc_I, 6 xd_I, 7 xd_J,
// each pre-scaled by its coefficient.  Per tile kind: (row-sum slice, column-sum slice,
// row output slot, column output slot) with slots 0 y1_I, 1 y1_J, 2 y2_I, 3 y2_J.
__device__ __forceinline__ void kind_roles(int kind, int& xr, int& xcs, int& orow, int& ocol) {
    switch (kind) {
        case 0: xr = 0; xcs = 6; orow = 0; ocol = 3; break;   // K_IJ: cK K x_a(J) -> y1_I; cT K^T x_d(I) -> y2_J
        case 1: xr = 1; xcs = 7; orow = 1; ocol = 2; break;   // K_JI: -> y1_J; -> y2_I
        case 2: xr = 2; xcs = 3; orow = 0; ocol = 1; break;   // V_IJ: cV V x_b(J) -> y1_I; cV V^T x_b(I) -> y1_J
        default: xr = 4; xcs = 5; orow = 2; ocol = 3; break;  // D_IJ: -> y2_I; -> y2_J
    }
}

template <int NV, int VAL>
__device__ __forceinline__ void butterfly(float (&v)[NV * VAL], int lane) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int off = 16 >> k;
        const int nv = (NV >> k) > 1 ? (NV >> k) : 1;
        if (nv > 1) {
            const bool up = (lane & off) != 0;
#pragma unroll
            for (int j = 0; j < nv / 2; ++j) {
#pragma unroll
                for (int q = 0; q < VAL; ++q) {
                    const float send = up ? v[j * VAL + q] : v[(j + nv / 2) * VAL + q];
                    const float keep = up ? v[(j + nv / 2) * VAL + q] : v[j * VAL + q];
                    v[j * VAL + q] = keep;
                    v[(j + nv / 2) * VAL + q] = __shfl_xor_sync(0xffffffffu, send, off);
                }
                if (VAL == 1) v[j] = __fadd_rn(v[j], v[j + nv / 2]);
                else dd_add(v[2 * j], v[2 * j + 1], v[2 * (j + nv / 2)], v[2 * (j + nv / 2) + 1]);
            }
        } else {
            float h[VAL];
#pragma unroll
            for (int q = 0; q < VAL; ++q) h[q] = __shfl_xor_sync(0xffffffffu, v[q], off);
            if (VAL == 1) v[0] = __fadd_rn(v[0], h[0]);
            else dd_add(v[0], v[1], h[0], h[1]);
        }
    }
}

template <class ST, int MODE, int R>
__global__ void __launch_bounds__(TP_THREADS, 1) k_tile(TileLaunch L) {
    using LT = Layout<ST, MODE, R>;
    using X = typename Arith<MODE>::X;
    using A = typename Arith<MODE>::A;
    constexpr int S = LT::S;
    constexpr int CH = Store<ST>::CHUNKS;
    constexpr int RPC = Store<ST>::RPC;
    constexpr int RPW = LT::RPW;
    constexpr int G = Group<R, RPW>::G;
    constexpr int NV = Group<R, RPW>::NV;
    constexpr int VAL = Arith<MODE>::VAL;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* stages = sm;
    X* xs = reinterpret_cast<X*>(sm + S * TP_CHUNK);                        // [8][R][64]
    A* acc = reinterpret_cast<A*>(sm + S * TP_CHUNK + LT::XS);              // [4][R][64]
    A* red = reinterpret_cast<A*>(sm + S * TP_CHUNK + LT::XS + LT::ACC);    // [8 warps][R][64]
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + S * TP_CHUNK + LT::XS + LT::ACC + LT::RED);
    uint64_t* empty = full + S;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mb_init(&full[i], 1);
            mb_init(&empty[i], TP_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == TP_WARPS) {  // ---------------------------------------------- producer
        if (lane == 0) {
            uint32_t q = 0;
            bool ok = true;
            for (int64_t k = blockIdx.x; k < L.items && ok; k += gridDim.x) {
                const ItemInfo it = decode_item(L.sets, L.nsets, k);
                int kinds[4];
                const unsigned char* src[4];
                const int ntl = item_tiles<ST>(L.sets[it.set], it.I, it.J, kinds, src);
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
    const X* __restrict__ xg = static_cast<const X*>(L.x);
    uint32_t q = 0;
    bool aborted = false;
    for (int64_t k = blockIdx.x; k < L.items; k += gridDim.x) {
        const ItemInfo it = decode_item(L.sets, L.nsets, k);
        const TileSet& St = L.sets[it.set];
        int kinds[4];
        const unsigned char* src[4];
        const int ntl = item_tiles<ST>(St, it.I, it.J, kinds, src);
        const bool diag = it.I == it.J;
        const int64_t N = St.N;
        // item start: input slices (scaled) and zeroed accumulators
        consumers_sync();
        for (int e = threadIdx.x; e < 8 * R * 64; e += 32 * TP_WARPS) {
            const int sl = e / (R * 64), r = (e / 64) % R, j = e % 64;
            const int tile = (sl == 0 || sl == 2 || sl == 4 || sl == 7) ? it.J : it.I;
            const int64_t off = sl < 2 ? St.xa : sl < 4 ? St.xb : sl < 6 ? St.xc : St.xd;
            const int ci = sl < 2 ? 0 : sl < 4 ? 1 : sl < 6 ? 2 : 3;
            const int64_t row = (int64_t)tile * 64 + j;
            X v{};
            if (r < L.rc && row < N && St.c[ci] != 0.0) {
                const X u = xg[(int64_t)r * L.n + off + row];
                if constexpr (MODE == TP_F32) {
                    const float c = St.ch[ci];
                    v = make_float2(c * u.x, c * u.y);
                } else {
                    // (u.hi + u.lo) (ch + cl) as a double-float pair per component
                    const float ch = St.ch[ci], cl = St.cl[ci];
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
            xs[e] = v;
        }
        for (int e = threadIdx.x; e < 4 * R * 64; e += 32 * TP_WARPS) acc[e] = A{};
        consumers_sync();
        for (int t = 0; t < ntl; ++t) {
            int sr_, sc_, orow, ocol;
            kind_roles(kinds[t], sr_, sc_, orow, ocol);
            const bool do_row = kinds[t] <= 1 ? St.c[0] != 0.0 : true;
            const bool do_col = kinds[t] <= 1 ? St.c[3] != 0.0 : !diag;
            if (diag) {
                orow = orow == 1 ? 0 : (orow == 3 ? 2 : orow);
                ocol = ocol == 1 ? 0 : (ocol == 3 ? 2 : ocol);
            }
            // row-sum inputs at the lane's two columns (registers)
            float xrh[R][2][2], xrl[R][2][2];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const X u = xs[(sr_ * R + r) * 64 + Store<ST>::col(lane, kk)];
                    xrh[r][kk][0] = u.x;
                    xrh[r][kk][1] = u.y;
                    if constexpr (MODE == TP_DD) {
                        xrl[r][kk][0] = u.z;
                        xrl[r][kk][1] = u.w;
                    } else {
                        xrl[r][kk][0] = xrl[r][kk][1] = 0.0f;
                    }
                }
            // column-sum partials of the lane's two columns
            float cp[R][2][2][VAL];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int w = 0; w < VAL; ++w) cp[r][kk][c][w] = 0.0f;
            const X* __restrict__ ycol = xs + sc_ * R * 64;
            for (int h = 0; h < CH; ++h, ++q) {
                const int st = (int)(q % S);
                if (!aborted && *abort_flag) aborted = true;
                if (!aborted && !mb_wait(&full[st], (q / S) & 1)) {
                    aborted = true;
                    if (lane == 0) atomicOr(L.err, 8);
                    *abort_flag = 1;
                }
                const unsigned char* chunk = stages + (size_t)st * TP_CHUNK;
#pragma unroll 1
                for (int g0 = 0; g0 < RPW; g0 += G) {
                    float v[NV * VAL];
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int lr = warp + TP_WARPS * (g0 + g);  // row within the chunk
                        const int i = h * RPC + lr;                  // row within the tile
                        float ah[4], al[4];
                        Store<ST>::load(chunk + (size_t)lr * Store<ST>::ROW_BYTES, lane, ah, al);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            // row sum of the lane's two entries
                            const int b = (g * R + r) * 2 * VAL;
                            if constexpr (MODE == TP_F32) {
                                float re = ah[0] * xrh[r][0][0];
                                re = fmaf(-ah[1], xrh[r][0][1], re);
                                re = fmaf(ah[2], xrh[r][1][0], re);
                                re = fmaf(-ah[3], xrh[r][1][1], re);
                                float im = ah[0] * xrh[r][0][1];
                                im = fmaf(ah[1], xrh[r][0][0], im);
                                im = fmaf(ah[2], xrh[r][1][1], im);
                                im = fmaf(ah[3], xrh[r][1][0], im);
                                v[b] = do_row ? re : 0.0f;
                                v[b + 1] = do_row ? im : 0.0f;
                            } else {
                                float rh = 0.0f, rl = 0.0f, ih = 0.0f, il = 0.0f;
                                if (do_row) {
                                    constexpr bool AL = Store<ST>::AL;
#pragma unroll
                                    for (int kk = 0; kk < 2; ++kk) {
                                        const float arh = ah[2 * kk], aih = ah[2 * kk + 1];
                                        const float arl = al[2 * kk], ail = al[2 * kk + 1];
                                        dd_mac<AL>(rh, rl, arh, arl, xrh[r][kk][0], xrl[r][kk][0]);
                                        dd_mac<AL>(rh, rl, -aih, -ail, xrh[r][kk][1], xrl[r][kk][1]);
                                        dd_mac<AL>(ih, il, arh, arl, xrh[r][kk][1], xrl[r][kk][1]);
                                        dd_mac<AL>(ih, il, aih, ail, xrh[r][kk][0], xrl[r][kk][0]);
                                    }
                                }
                                v[b] = rh;
                                v[b + 1] = rl;
                                v[b + 2] = ih;
                                v[b + 3] = il;
                            }
                            // column sums: the lane's entries times the column input of row i
                            if (do_col) {
                                const X y = ycol[r * 64 + i];
                                if constexpr (MODE == TP_F32) {
#pragma unroll
                                    for (int kk = 0; kk < 2; ++kk) {
                                        const float ar = ah[2 * kk], ai = ah[2 * kk + 1];
                                        cp[r][kk][0][0] = fmaf(ar, y.x, fmaf(-ai, y.y, cp[r][kk][0][0]));
                                        cp[r][kk][1][0] = fmaf(ar, y.y, fmaf(ai, y.x, cp[r][kk][1][0]));
                                    }
                                } else {
                                    constexpr bool AL = Store<ST>::AL;
#pragma unroll
                                    for (int kk = 0; kk < 2; ++kk) {
                                        const float arh = ah[2 * kk], aih = ah[2 * kk + 1];
                                        const float arl = al[2 * kk], ail = al[2 * kk + 1];
                                        dd_mac<AL>(cp[r][kk][0][0], cp[r][kk][0][1], arh, arl, y.x, y.z);
                                        dd_mac<AL>(cp[r][kk][0][0], cp[r][kk][0][1], -aih, -ail, y.y, y.w);
                                        dd_mac<AL>(cp[r][kk][1][0], cp[r][kk][1][1], arh, arl, y.y, y.w);
                                        dd_mac<AL>(cp[r][kk][1][0], cp[r][kk][1][1], aih, ail, y.x, y.z);
                                    }
                                }
                            }
                        }
                    }
                    if (do_row) {
                        butterfly<NV, VAL>(v, lane);
                        // the lane pair (2 qv, 2 qv + 1) holds value qv = (g R + r) 2 + re/im
                        constexpr int SH = NV >= 32 ? 0 : (NV >= 16 ? 1 : (NV >= 8 ? 2 : (NV >= 4 ? 3 : (NV >= 2 ? 4 : 5))));
                        const int qv = (lane >> SH) & (NV - 1);
                        if ((lane & ((1 << SH) - 1)) == 0) {
                            const int comp = qv & 1, rr = (qv >> 1) % R, g = (qv >> 1) / R;
                            const int i = h * RPC + warp + TP_WARPS * (g0 + g);
                            float* a = reinterpret_cast<float*>(&acc[(orow * R + rr) * 64 + i]);
                            if constexpr (MODE == TP_F32) {
                                a[comp] = __fadd_rn(a[comp], v[0]);
                            } else {
                                dd_add(a[comp], a[2 + comp], v[0], v[1]);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mb_arrive(&empty[st]);
            }
            if (do_col) {  // the eight warps' column partials into the output slot
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        A a;
                        if constexpr (MODE == TP_F32) a = make_float2(cp[r][kk][0][0], cp[r][kk][1][0]);
                        else a = make_float4(cp[r][kk][0][0], cp[r][kk][1][0], cp[r][kk][0][1], cp[r][kk][1][1]);
                        red[(warp * R + r) * 64 + Store<ST>::col(lane, kk)] = a;
                    }
            }
            consumers_sync();
            if (do_col) {
                for (int e = threadIdx.x; e < R * 64; e += 32 * TP_WARPS) {
                    A s = red[e];
#pragma unroll
                    for (int w = 1; w < TP_WARPS; ++w) {
                        const A b = red[w * R * 64 + e];
                        if constexpr (MODE == TP_F32) {
                            s.x = __fadd_rn(s.x, b.x);
                            s.y = __fadd_rn(s.y, b.y);
                        } else {
                            dd_add(s.x, s.z, b.x, b.z);
                            dd_add(s.y, s.w, b.y, b.w);
                        }
                    }
                    A& d = acc[ocol * R * 64 + e];
                    if constexpr (MODE == TP_F32) {
                        d.x = __fadd_rn(d.x, s.x);
                        d.y = __fadd_rn(d.y, s.y);
                    } else {
                        dd_add(d.x, d.z, s.x, s.z);
                        dd_add(d.y, d.w, s.y, s.w);
                    }
                }
            }
            consumers_sync();
        }
        // item end: the output slices into their partial-sum slots
        const bool y1 = St.y1 >= 0, y2 = St.y2 >= 0;
        const int64_t nt = St.nt;
        for (int e = threadIdx.x; e < 4 * R * 64; e += 32 * TP_WARPS) {
            const int slot = e / (R * 64), r = (e / 64) % R, row = e % 64;
            if (diag && (slot == 1 || slot == 3)) continue;
            if ((slot < 2 && !y1) || (slot >= 2 && !y2) || r >= L.rc || aborted) continue;
            const int out = slot >> 1;
            const int64_t trow = (slot & 1) ? it.J : it.I, tcol = (slot & 1) ? it.I : it.J;
            const int64_t idx = St.part * R + ((((out * nt + trow) * nt + tcol) * R + r) << 6) + row;
            static_cast<A*>(L.part)[idx] = acc[e];
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
    using LT = Layout<ST, MODE, R>;
    BEM_CUDA_TRY(cudaFuncSetAttribute(k_tile<ST, MODE, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, LT::BYTES));
    int dev = 0, sms = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TileLaunch L;
    L.sets = P.dsets.as<TileSet>();
    L.nsets = (int)P.sets.size();
    L.rc = rc;
    L.items = P.items;
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
    BEM_LAUNCH_PTR(names[sizeof(ST) == 16][MODE][ri], (k_tile<ST, MODE, R>), grid, TP_THREADS, LT::BYTES, s, L);
    static const char* rnames[2][4] = {
        {"k_tile_reduce<f32,1>", "k_tile_reduce<f32,2>", "k_tile_reduce<f32,4>", "k_tile_reduce<f32,8>"},
        {"k_tile_reduce<dd,1>", "k_tile_reduce<dd,2>", "k_tile_reduce<dd,4>", "k_tile_reduce<dd,8>"}};
    BEM_LAUNCH_PTR(rnames[MODE][ri], (k_tile_reduce<MODE, R>), dim3((unsigned)P.rtiles, (unsigned)rc),
                   64 * RED_GROUPS, 0, s, L.sets, L.nsets, P.rtiles, P.n, part, z);
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
    BEM_TRY(P.dsets.alloc(P.sets.size() * sizeof(TileSet), s));
    BEM_CUDA_TRY(cudaMemcpyAsync(P.dsets.p, P.sets.data(), P.sets.size() * sizeof(TileSet), cudaMemcpyHostToDevice, s));
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
            case 4: return launch_tile<float2, TP_DD, 4>(P, rc, x, z, part, err, s);
            default: return launch_tile<float2, TP_DD, 8>(P, rc, x, z, part, err, s);
        }
    }
    switch (R) {
        case 1: return launch_tile<double2, TP_DD, 1>(P, rc, x, z, part, err, s);
        case 2: return launch_tile<double2, TP_DD, 2>(P, rc, x, z, part, err, s);
        case 4: return launch_tile<double2, TP_DD, 4>(P, rc, x, z, part, err, s);
        default: return launch_tile<double2, TP_DD, 8>(P, rc, x, z, part, err, s);
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
