// Internal declarations of the GB300 transmission-BEM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/bem.h"

namespace bem {

inline double now_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ autotuner table
// Launch shapes chosen by bem_autotune (tune.cu): per kernel family, width (columns per
// launch) and size class ceil(log2(rows)), a block size and a variant.
enum { TUNE_GEMM_TC = 0, TUNE_CHEB = 1, TUNE_KERNELS = 2 };
struct TuneChoice {
    int block;    // threads per block (0: the kernel's own)
    int variant;  // gemm_tc: K splits (1 or 2); cheb: 0
    double ms;    // time measured for it
};
int size_class(int64_t n);
TuneChoice tune_get(int kernel, int width, int64_t n, TuneChoice dflt);
void tune_put(int kernel, int width, int64_t n, TuneChoice c);
inline bool tune_choice_valid(int kernel, const TuneChoice& c) {
    switch (kernel) {
        case TUNE_GEMM_TC: return c.block == 0 && (c.variant == 1 || c.variant == 2);
        case TUNE_CHEB: return (c.block == 64 || c.block == 128 || c.block == 256) && c.variant == 0;
        default: return false;
    }
}

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);

#define BEM_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ::bem::set_error(std::string("CUDA error ") + cudaGetErrorString(e_) +  \
                             " at " __FILE__ ":" + std::to_string(__LINE__) +       \
                             " in " #expr);                                         \
            return e_ == cudaErrorMemoryAllocation ? BEM_E_OOM : BEM_E_CUDA;        \
        }                                                                           \
    } while (0)

#define BEM_CHECK_LAUNCH() BEM_CUDA_TRY(cudaGetLastError())

// Number of kernels this library has launched since it was loaded (a CUDA graph launch
// counts its kernel nodes).
void count_launch(uint64_t n = 1);

// Nonzero while this thread records launches into a CUDA graph (stream capture): they
// are then neither timed nor counted (the graph's launches are counted instead).
extern thread_local int g_capturing;

// Optional per-kernel event timing (profile.cu); -1 when profiling is off.
int prof_begin(const char* name, cudaStream_t s);
void prof_end(int slot, cudaStream_t s);
// True while profiling times every kernel (no selection): fixed launch sequences are
// then launched kernel by kernel instead of as CUDA graphs, so that each is timed.
bool prof_times_every_kernel();

// Launch a kernel, time it when profiling is on, count it and check the launch.
#define BEM_LAUNCH(kern, grid, block, smem, stream, ...)                \
    do {                                                                \
        const int prof_slot_ =                                          \
            ::bem::g_capturing ? -1 : ::bem::prof_begin(#kern, (stream)); \
        kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);       \
        ::bem::prof_end(prof_slot_, (stream));                          \
        if (!::bem::g_capturing) ::bem::count_launch();                 \
        BEM_CHECK_LAUNCH();                                             \
    } while (0)

// The same for a kernel given as a function pointer (a template instance chosen at run
// time), timed by the profiler under `name`.
#define BEM_LAUNCH_PTR(name, kptr, grid, block, smem, stream, ...)       \
    do {                                                                \
        const int prof_slot_ =                                          \
            ::bem::g_capturing ? -1 : ::bem::prof_begin((name), (stream)); \
        (kptr)<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);     \
        ::bem::prof_end(prof_slot_, (stream));                          \
        if (!::bem::g_capturing) ::bem::count_launch();                 \
        BEM_CHECK_LAUNCH();                                             \
    } while (0)

#define BEM_TRY(expr)                      \
    do {                                   \
        bem_status s_ = (expr);            \
        if (s_ != BEM_OK) return s_;       \
    } while (0)

#define BEM_REQUIRE(cond, msg)                                   \
    do {                                                         \
        if (!(cond)) {                                           \
            ::bem::set_error(std::string("invalid argument: ") + (msg)); \
            return BEM_E_INVALID_ARG;                            \
        }                                                        \
    } while (0)

// ------------------------------------------------------------------ device buffers
// Stream-ordered device allocation owned by RAII handles.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
    DevBuf& operator=(DevBuf&& o) noexcept {
        release();
        p = o.p; bytes = o.bytes; stream = o.stream;
        o.p = nullptr; o.bytes = 0;
        return *this;
    }
    ~DevBuf() { release(); }
    bem_status alloc(size_t nbytes, cudaStream_t s);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------------ quadrature
// 6-point degree-4 symmetric triangle rule on {s,t >= 0, s+t <= 1}, weights sum 1/2.
struct TriRule {
    double s[6], t[6], w[6];
};
const TriRule& tri_rule_degree4();

// Sauter-Schwab tables: points (x1, x2, y1, y2) on T^ x T^ with T^ = {0<=x2<=x1<=1},
// weight including the transformation Jacobian.  kind: 0 coincident, 1 edge, 2 vertex.
struct SSTable {
    int n = 0;                 // Gauss points per axis
    int count[3] = {0, 0, 0};  // points per kind
    int offset[3] = {0, 0, 0};
    std::vector<double> host;  // [total][5]
    DevBuf dev;
};
bem_status ss_table_get(int n, cudaStream_t stream, const double** dev_ptr, int count[3], int offset[3]);

// ------------------------------------------------------------------ geometry record
// Per-triangle record, 50 doubles (400 bytes), written by the geometry kernel.
struct __align__(16) TriRec {
    double q[6][3];    // physical quadrature points             (doubles  0..17)
    double wl[6][3];   // w_p * J * lambda_a(p)                  (doubles 18..35)
    double n[3];       // outward unit normal                    (doubles 36..38)
    double J;          // |e1 x e2|                              (double  39)
    double curl[3][3]; // surface curls of the shape functions   (doubles 40..48)
    double pad;
};
constexpr int TRIREC_DOUBLES = 50;
static_assert(sizeof(TriRec) == TRIREC_DOUBLES * 8, "TriRec layout");

// FP32 per-triangle record of the mixed-precision assembly (56 floats, 224 bytes),
// stored in tile order.  The centroid is a double-float pair (hi + lo); quadrature
// points are stored relative to the centroid so that FP32 keeps them accurate.
struct __align__(16) TriRec32 {
    float ch[3], cl[3];  // centroid, hi and lo parts             (floats  0..5)
    float u[6][3];       // quadrature points minus the centroid  (floats  6..23)
    float wl[6][3];      // w_p * J * lambda_a(p)                 (floats 24..41)
    float n[3];          // outward unit normal                   (floats 42..44)
    float curl[3][3];    // surface curls                         (floats 45..53)
    float pad[2];
};
constexpr int TRIREC32_FLOATS = 56;
static_assert(sizeof(TriRec32) == TRIREC32_FLOATS * 4, "TriRec32 layout");

// Tiles of the mixed-precision assembly: at most TILE_TRI triangles and at most
// TILE_NV distinct vertices each.
constexpr int TILE_TRI = 32;
constexpr int TILE_NV = 40;

// Singular pair: kind 1 edge / 2 vertex, triangles t < s, Sauter-Schwab vertex order.
struct SingPair {
    int32_t t, s;
    uint8_t pt[3], ps[3];
    uint8_t kind, pad;
};

}  // namespace bem

// ------------------------------------------------------------------ handles
struct bem_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // stop request checked by the solver between GMRES iterations (serving)
    const std::atomic<int>* cancel = nullptr;
    double deadline = 0.0;  // steady-clock seconds; 0 = none
    // set by the caller when its solves never overlap with others on the device: the
    // mass inverses then run as one cooperative launch with grid barriers (off by
    // default: measured no faster than the step launches replayed as CUDA graphs)
    bool exclusive = false;
};

struct bem_grid {
    bem_context* ctx = nullptr;
    int64_t nv = 0, nt = 0;
    std::vector<double> h_xyz;     // host copy (intake)
    std::vector<int32_t> h_tri;
    bem::DevBuf xyz, tri, rec;     // device: vertices, triangles, TriRec per triangle
    // singular pairs (edge and vertex-adjacent, unordered t < s)
    bem::DevBuf sing;
    int64_t n_edge = 0, n_vertex = 0;
    // mass matrix CSR structure (rows = vertices) and per-triangle slot map
    bem::DevBuf m_rowptr, m_col, m_slot;   // m_slot [nt][3][3] CSR position
    int64_t m_nnz = 0;
    int32_t m_maxrow = 0;                  // largest number of entries in a mass row
    double surface_area = 0.0;
    // tiles of the mixed-precision assembly (triangles in tile order)
    int64_t ntile = 0;
    bem::DevBuf t_order;        // tile position -> triangle index           [nt]
    bem::DevBuf t_verts;        // vertex ids of triangles in tile order     [nt][3]
    bem::DevBuf t_slots;        // local vertex slots in the tile, 3 bytes   [nt]
    bem::DevBuf tile_tstart;    // first tile position of each tile          [ntile + 1]
    bem::DevBuf tile_vstart;    // first entry of each tile's vertex list    [ntile + 1]
    bem::DevBuf tile_vert;      // tile vertex lists (global vertex ids)
    bem::DevBuf rec32;          // TriRec32 in tile order                    [nt]
};

struct bem_matrix {
    int64_t rows = 0, cols = 0;
    int entry_bytes = 16;          // 16: complex128, 8: complex64
    bem::DevBuf data;              // row-major
};

struct bem_sparse {
    int64_t rows = 0, cols = 0, nnz = 0;
    bem::DevBuf row, col, val;     // COO, int32 / int32 / double
};

namespace bem {

// ------------------------------------------------------------------ operator storage
// Dense operators of one grid as 64 x 64 tiles, each tile contiguous (row-major
// inside, 64 x 64 entries) so that a whole tile is one bulk copy:
//   OP_FULL: all nt x nt tiles, tile (I, J) at index I nt + J (K);
//   OP_SYM:  a symmetric matrix (V, D) keeps only the tiles I <= J, in row-major order
//            of the upper tile triangle, tile (I, J) at index I nt - I (I - 1) / 2 + (J - I);
//            diagonal tiles hold both halves.  Entry (i, j) of a lower tile is entry
//            (j, i) of its mirror.
//   OP_DENSE: plain row-major N x N (bem_assemble's result).
// T = K^T is never stored: products apply K in both orientations.  Rows and columns
// past N in the last tile row / column are zero.
constexpr int OPT = 64;
enum : int { OP_DENSE = 0, OP_FULL = 1, OP_SYM = 2 };
__host__ __device__ inline int op_tiles(int64_t N) { return (int)((N + OPT - 1) / OPT); }
__host__ __device__ inline int64_t op_sym_tile(int64_t I, int64_t J, int64_t nt) {
    return I * nt - I * (I - 1) / 2 + (J - I);
}
inline size_t op_entries(int layout, int64_t N) {
    const size_t nt = (size_t)op_tiles(N);
    return layout == OP_DENSE ? (size_t)N * N : layout == OP_FULL ? nt * nt * OPT * OPT : nt * (nt + 1) / 2 * OPT * OPT;
}
// storage index of entry (i, j), or -1 where a symmetric layout keeps its mirror instead
__host__ __device__ inline int64_t op_index(int layout, int64_t N, int nt, int64_t i, int64_t j) {
    if (layout == OP_DENSE) return i * N + j;
    const int64_t I = i >> 6, J = j >> 6;
    const int64_t in = ((i & 63) << 6) | (j & 63);
    if (layout == OP_FULL) return ((I * nt + J) << 12) | in;
    if (I > J) return -1;
    return (op_sym_tile(I, J, nt) << 12) | in;
}
// storage layouts of (V, K, T, D) in a product-ready operator set and in bem_assemble
struct OpLayouts {
    int lay[4];
};
inline OpLayouts op_layouts_tiled() { return OpLayouts{{OP_SYM, OP_FULL, OP_FULL, OP_SYM}}; }
inline OpLayouts op_layouts_dense() { return OpLayouts{{OP_DENSE, OP_DENSE, OP_DENSE, OP_DENSE}}; }

// ------------------------------------------------------------------ tile products
// One grid's operators in one product (tile_product.cu):
//   y1 = cK K xa + cV V xb,   y2 = cD D xc + cT K^T xd
// with K, V, D tiled (OP_FULL, OP_SYM, OP_SYM; complex64 or complex128 by the product's
// storage), x and z columns of n entries, the inputs at offsets xa..xd of a column and
// the outputs written at offsets y1, y2 (-1: not computed).  A zero coefficient (or a
// null matrix) skips that matrix's bytes altogether.
struct TileSet {
    const void* K;
    const void* V;
    const void* D;
    int64_t N;
    int32_t nt;
    int32_t flags;          // TS_* bits: the matrices and outputs this set uses
    double c[4];            // cK, cV, cD, cT
    float ch[4], cl[4];     // the same as double-float pairs (high, low)
    int64_t xa, xb, xc, xd;
    int64_t y1, y2;
    int64_t item0;          // first work item of this set in the launch (items: tile pairs I <= J)
    int64_t rtile0;         // first output row tile (2 nt per set)
    int64_t part;           // element offset of this set's partial sums (per column)
};
enum : int { TS_KROW = 1, TS_KCOL = 2, TS_V = 4, TS_D = 8, TS_Y1 = 16, TS_Y2 = 32 };
enum : int { TP_F32 = 0, TP_DD = 1 };  // arithmetic: FP32 on complex64; double-float (FP64-accurate)
struct TileProd {
    std::vector<TileSet> sets;
    DevBuf dsets;            // device copy of sets
    DevBuf ditems;           // work items: int2 (set, I << 16 | J), in set order
    int64_t items = 0, rtiles = 0, part_per_col = 0;
    int64_t n = 0;           // column length of x and z
    int storage = 8;         // bytes per matrix entry: 8 (complex64) or 16 (complex128)
};
// add a set (coefficients cK, cV, cD, cT; offsets) to a product under construction
void tile_prod_add(TileProd& P, const void* K, const void* V, const void* D, int64_t N, double cK, double cV,
                   double cD, double cT, int64_t xa, int64_t xb, int64_t xc, int64_t xd, int64_t y1, int64_t y2);
// upload the sets (once; the product is then reused with any inputs)
bem_status tile_prod_finish(TileProd& P, int64_t n, int storage, cudaStream_t s);
// bytes of partial sums one product of R columns needs
size_t tile_part_bytes(const TileProd& P, int mode, int R);
// z (rc <= 8 columns of n) = the product applied to x: complex64 x (float2) in TP_F32,
// double-float x (float4: re hi, im hi, re lo, im lo) in TP_DD.  part: tile_part_bytes.
bem_status tile_product(const TileProd& P, int mode, int rc, const void* x, double2* z, void* part, int* err,
                        cudaStream_t s);
// dense row-major copy of a tiled operator (transpose: K^T, i.e. T, from K's tiles)
bem_status tiles_to_dense(const void* src, int layout, bool transpose, int64_t N, int storage, void* dst,
                          cudaStream_t s);
// seeded random operators of an N-vertex grid in the tiled storage (tiles: V, K, D) and,
// if dense is not null, their dense row-major copies (dense: V, K, T, D)
bem_status random_tiled_ops(int64_t N, int storage, uint64_t seed, DevBuf tiles[3], DevBuf* dense, cudaStream_t s);
// self-test: tile products on seeded random operators against an FP64 dense product
// (max relative error over the outputs)
bem_status selftest_tile(int mode, int storage, int R, double* rel_err, cudaStream_t s);

// grid.cu
bem_status grid_build_geometry(bem_grid* g);
bem_status mass_values(const bem_grid* g, double* d_val, cudaStream_t s);      // [m_nnz]
bem_status mass_inverse_diag(const bem_grid* g, const double* d_val, double* d_dinv, cudaStream_t s);

// grid.cu: FP32 geometry records in tile order (mixed-precision assembly)
bem_status grid_build_rec32(const bem_grid* g, cudaStream_t s);

// assemble32.cu: regular pairs in FP32 into complex64 V, K, T, D (layouts L; zeroed by the caller)
bem_status assemble_regular_fp32(const bem_grid* g, double k_re, double k_im, float2* V, float2* K, float2* T,
                                 float2* D, const OpLayouts& L, cudaStream_t s);
// assemble32.cu: accuracy self-test of the FP32 kernel's sincos against CUDA's sincosf
bem_status selftest_sincos(int n, float xmax, double* max_err, cudaStream_t s);
// assemble.cu: singular pairs (FP64 quadrature) added into complex64 matrices (layouts L)
bem_status assemble_singular_into_c64(const bem_grid* g, double k_re, double k_im, int n_singular, float2* V,
                                      float2* K, float2* T, float2* D, const OpLayouts& L, cudaStream_t s);

// assemble.cu: V, K, T, D (complex128 in layouts L, zeroed here; any pointer may be null).
bem_status assemble_operators_fp64(const bem_grid* g, double k_re, double k_im, int n_singular,
                                   double2* V, double2* K, double2* T, double2* D, const OpLayouts& L,
                                   cudaStream_t s);

// mortar.cu: COO of P_ab (rows: vertices of a, cols: vertices of b).
// FP32 regular pairs of many grids in one persistent launch (assemble32.cu)
bem_status assemble_regular_fp32_many(int count, const bem_grid* const* g, const double* k_re, const double* k_im,
                                      float2* const* V, float2* const* K, float2* const* T, float2* const* D,
                                      const OpLayouts& L, cudaStream_t s);

// tensor-core multi-column MTF product (gemm_tc.cu)
int tc_padded_columns(int R);
size_t tc_workspace_bytes(const int64_t N[4], int RP);
bem_status mtf_product_tc(const float2* const a1[4], const float2* const a2[4], const double c1[4],
                          const double c2[4], const int64_t N[4], const int64_t base[4], const int64_t x1[4],
                          const int64_t x2[4], int64_t n, int R, const double2* x, double2* z, void* work,
                          size_t work_bytes, int* err, cudaStream_t s);
bem_status selftest_tc(int R, double* rel_err, cudaStream_t s, int kind = 1);  // 1 TF32, 2 FP16, 3 BF16

// FP16-split tensor-core product fed by TMA (gemm_tc16.cu): the operator copy of the
// four block rows ([A1 | A2] rows as FP16 hi / lo parts, scaled by 2^eA, padded to Kp)
struct Tc16Ops {
    DevBuf hi[4], lo[4];
    int64_t N[4] = {0, 0, 0, 0}, Kp[4] = {0, 0, 0, 0};
    int eA[4] = {0, 0, 0, 0};
    bool bf16 = false;  // BF16 parts instead of FP16
};
bem_status tc16_build(const float2* const a1[4], const float2* const a2[4], const int64_t N[4], Tc16Ops& out,
                      cudaStream_t s, bool bf16 = false);
size_t tc16_workspace_bytes(const int64_t N[4], int RP);
bem_status mtf_product_tc16(const Tc16Ops& ops, const double c1[4], const double c2[4], const int64_t base[4],
                            const int64_t x1[4], const int64_t x2[4], int64_t n, int R, const double2* x,
                            double2* z, void* work, size_t work_bytes, int* err, cudaStream_t s);
bem_status selftest_barrier(double* result, cudaStream_t s);

bem_status mortar_coo(const bem_grid* a, const bem_grid* b, const double center[3],
                      DevBuf& row, DevBuf& col, DevBuf& val, int64_t* nnz, cudaStream_t s);

// Many transmission instances in lockstep (solver.cu).  Instances with the same grids
// and wavenumbers share one copy of their operators, masses and mortar.  halt (may be
// null) is asked, for each running instance, between GMRES iterations: a status other
// than BEM_OK stops that instance alone (cancellation, deadlines); status_out[count]
// (may be null) receives each instance's outcome.
using HaltCheck = std::function<bem_status(int)>;
bem_status solve_many_impl(bem_context* ctx, int count, const bem_instance* inst, const bem_solve_opts* o,
                           int on_device, bem_solve_report* reps, const HaltCheck* halt = nullptr,
                           int32_t* status_out = nullptr);

}  // namespace bem
