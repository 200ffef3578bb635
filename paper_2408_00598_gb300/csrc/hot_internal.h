// Device-side data structures shared by the HOT kernels and the host engine.
//
// Layout of one instance (an m x n grid) in device memory.  The flow vector
// x = [f1; f2] of the reduced model (eq. 3-4 of arXiv 2408.00598) is stored as
// n + m "slabs", slab-major, row-major inside a slab:
//   slab s <  n : f1 for column j = s;      m x m, row = k, col = i   (f1_{i,k,j})
//   slab s >= n : f2 for row    k = s - n;  n x n, row = j, col = l   (f2_{k,j,l})
// (offsets in the g_* helpers below).  In both halves the cost is
// (X_r - X_c)^2 with X the bin coordinates of that axis (eq. 4), A^T y at
// (s, r, c) is alpha_s[r] + beta_s[c] with
//   f1 slab j: alpha[k] =  y1(k,j), beta[i] = y2(i,j)
//   f2 slab k: alpha[j] = -y1(k,j), beta[l] = y3(k,l)   (y3(m-1,n-1) = 0),
// and the row and column sums of a slab are the A x products:
//   (A x)_1(k,j) = rowsum(f1 slab j)[k] - rowsum(f2 slab k)[j]
//   (A x)_2(i,j) = colsum(f1 slab j)[i]
//   (A x)_3(k,l) = colsum(f2 slab k)[l]        ((m-1,n-1) row dropped, eq. 7-8)
// Every reduction of the method is therefore slab-local.
//
// The iterate is kept in the reduced form v = x + sigma z (the shadow sequence
// of App. A): the Halpern anchor v0 and the delta d = v - v0.  The anchor is
// stored relative to sigma times its own reduced cost, u = v0 - sigma g0 with
// g0 = c - A^T y0 (y0 the dual of the restart point), so every stored and
// computed per-element quantity is small where the iteration cancels:
//   v / sigma  = g0 + (u + d) / sigma,
//   g - v/sigma = -A^T(y - y0) - (u + d)/sigma,
//   x-bar      = u + d + sigma A^T(y - y0).
// The same iterate, exactly; only the rounding of FP32 storage changes.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hot {

constexpr int kThreads = 256;          // block size of the tile kernels
constexpr int kNK = 5;                 // per-tile check partials: r^2, min^2, x^2, z^2, c.x
constexpr int kRowSmemBytes = 16384;   // row-partial buffer of a sweep tile
constexpr int kMaxS = 1024;
constexpr int kAPT = 4;                // k_alpha32: pieces per thread and chunk
constexpr int kAlphaChunk = kThreads * kAPT;
constexpr int kMaxTR = 128;            // FP32 tiles: TR * max(m, n) <= kRowSmemBytes / 4
constexpr int kMaxTileElems = 16384;   // FP32 tiles: TR * (longer row pitch) <= this

enum : int {
    ST_RUNNING = 0,
    ST_CONVERGED = 1,
    ST_CAPPED = 2,
    ST_NUMERIC = 3,
    ST_CANCELLED = 4,
};

// Per-instance control block, mutated only by the block-end kernels
// (k_check, k_restart_sigma, k_block_end) and read by every kernel.
struct HotCtl {
    double sigma;          // current sigma
    double tol;            // relative KKT tolerance
    double r0, rprev;      // restart residuals of the current cycle (< 0: unset)
    double rel_kkt, rel_dual, rel_comp, rel_primal;
    double abs_kkt;        // max of the three KKT terms without normalisers
    double pobj, dobj;     // unscaled primal <c,x-bar> and dual <b,y-bar>
    double dx2, dz2;       // ||x-bar - x_r||^2, ||z-bar - z_r||^2 at the last restart
    double sigma_old;      // sigma of the check iteration that triggered the last restart
    double res_norm;       // ||w - w-bar||_M at the last check
    long long total;       // iterations completed before the current block
    long long max_iter;
    int k;                 // Halpern counter at the start of the block
    int status;            // ST_*
    int restarts;
    int restart_pending;   // set at a check, consumed by the restart kernels
    int just_finished;     // set at the check that ends the solve
    int cancel;            // host asks the instance to stop at the next check
    unsigned int ymax_bits;// max |alpha|, |beta| (float bits, scaled units)
    int dzero;             // FP32: a restart left the delta zero (not stored); the
                           // next block's first sweep reads no d (cleared at the check)
};

// Element constants of one iteration in FP32 mode (formed once per instance
// and iteration by k_alpha32 from sigma and the Halpern counter).
struct P32 {
    float sih;        // 1/sigma
    float sf;         // sigma
    float rho, trs;   // Halpern: rho = (k+1)/(k+2), trs = 2 rho sigma
    float h;          // 2^-E
    float pad[3];
};

// Prop. 3 constants that change only with sigma, i.e. once per cycle, as
// double-float pairs (FP32 mode): 1/sigma, 1/n, 1/m, 1/(m+n), 1/m + 1/n,
// 1/w, the last diagonal entry dl of W-hat, the sum of its diagonal,
// 1/(sigma m), 1/(sigma n), and mu2(m,n) minus the anchor's column total
// there (the dropped row of eq. 7).  Written by k_anchor, read by k_alpha32.
struct CycleK {
    float2 is, in, im, imn, imin, iw, dl, sumd, isim, isin, mk, pad;
};

// Per-instance descriptor (read-only while a block runs).
struct HotInst {
    int m, n;              // grid: mu is m x n (rows i/k, columns j/l)
    int mp, np;            // row pitches of the f1 (side m) and f2 (side n) slabs: the side rounded up to a multiple of 4
    int E;                 // cost scale 2^E >= max c; scaled cost = c * 2^-E
    int TR;                // rows per sweep tile
    int nb1, nb2;          // bands (tiles) per f1 slab = ceil(m / TR), per f2 slab = ceil(n / TR)
    int n_k1;              // chunks of the A x - b kernel
    int n_achunk;          // chunks of k_alpha32 (kAlphaChunk pieces each; FP32 mode)
    int fp64;              // 1: FP64 state, 0: FP32 anchor + delta
    int gadmm;             // 1: Step 4 of the generalized ADMM instead of Halpern's
    int stop_abs;          // 1: stop on the absolute KKT residual
    int coord_real;        // FP32 mode: some bin coordinate is not an integer in [-2048, 2048], so the
                           // pieces carry h x^2 - alpha as pairs and the sweep forms the cost term in pairs
    double relax;          // rho of the generalized ADMM
    double h;              // 2^-E
    double norm_b;         // ||b||
    double norm_c;         // ||c|| of the scaled problem
    double sum_mu1;        // sum of mu1 (1 within 1e-9), the column totals' sum
    double sum_mu2;        // sum of mu2 over every entry (the dropped one included)
    // per-instance arrays, sized for the slab layout: V = mn(m + n) flow
    // variables; "per slab row" arrays hold 2mn entries (g_row), "pieces" 4mn
    // (alpha then beta of each slab), column partials one row per band (g_colp)
    void* u;               // anchor, reduced: u = v0 - sigma (c - A^T y0)   [V]
    void* d0;              // delta, ping             [V]
    void* d1;              // delta, pong             [V]
    void* xr;              // x-bar at the last restart (final x-bar after the solve)
    void* zr;              // z-bar at the last restart
    float4* ab32;          // [4mn] pieces (hi, lo, delta, x) of alpha then beta, x the row/column coordinate, FP32 mode
    float2* ab0_32;        // [4mn] (hi, lo) split of ab0, FP32 mode (fixed within a cycle)
    double* ab64;          // [4mn] alpha then beta = A^T y-bar pieces (FP64 mode)
    double* ab0;           // [4mn] the same pieces of A^T y0 at the anchor
    double* dab64;         // [4mn] A^T (y-bar - y0) pieces
    double* rs;            // [2mn] row sums of the delta written by the last sweep
    double* cs_part;       // [slab][band][column] partial sums of the delta (FP64 mode)
    float* cs32;           // [slab][band][column] partial sums of the delta (FP32 mode)
    double* R1a;           // [2mn] anchor part of R1 along each slab's rows: -(rowsum f1 - rowsum f2)(u)/sigma
    double* kapa;          // [2mn] column totals of u per slab
    double* rs0;           // [2mn] row sums of u (FP64)
    double* cs0_part;      // [slab][band][column] partial sums of u
    double* xrs;           // [2mn] row sums of x-bar (check iterations)
    double* xcs_part;      // [slab][band][column] partial sums of x-bar
    double* tile_kkt;      // [tiles][kNK], tiles = n nb1 + m nb2
    double* rst_part;      // [tiles][2]
    double* vecs;          // [4][max(m, n)]: T1, T2, P1, P2 (slab totals and cross-slab row sums)
    double* mvec;          // [4][max(m, n)]: instance-wide vectors of Prop. 3 (k_marg)
    double* mu1;           // [m][n] row-major mu1(i, j)
    double* mu2;           // [m][n] row-major mu2(k, l)
    double* colmu1;        // [n] sum_i mu1(i, j)
    double* rowmu2;        // [m] sum_l mu2(k, l)
    double* k1_part;       // [n_k1] partial ||A x - b||^2
    double* dobj_part;     // partial <b, y>: [m + n] per slab (FP64 mode), [n_achunk] per chunk (FP32 mode)
    double* cu_part;       // [tiles] <c, u> per tile (FP32 mode, set per cycle)
    double* cD_part;       // [n_achunk] <c, A^T(y-bar - y0)> per k_alpha32 chunk (FP32 mode, check iterations)
    // FP32 bulk mode only (null in FP64 mode): the per-iteration Prop. 3
    // arithmetic runs on double-float pairs (hi, lo) of FP32 values, whose
    // sum carries about 48 significant bits, instead of FP64
    float2* rs2;           // [2mn] row sums of u + d (last sweep; = rs02 after a restart)
    float2* rs02;          // [2mn] row sums of u (fixed within a cycle)
    float2* K2;            // [2mn] (mu - colsum u)/(sigma m) per slab column (/(sigma n) for f2), fixed within a cycle
    float2* vec2;          // rows of max(m, n): T1, T2, then ceil(n/64) partials of P1 and ceil(m/64) of P2, of u + d
    float2* dab2;          // [4mn] pieces of A^T(y-bar - y0)
    float2* stg2;          // [4][max(m, n)] Prop. 3 stage of the current iteration: mvA, mvS, sy, sp (k_stage32)
    unsigned int* vcount;  // k_vec32 items of this instance finished in the running launch (0 between launches)
    float2* mu1f;          // [m][n] mu1 as pairs
    float2* mu2f;          // [m][n] mu2 as pairs
    float2* cm2;           // [n] colmu1 as pairs
    float2* rm2;           // [m] rowmu2 as pairs
    P32* p32;              // element constants of the current iteration
    const float* X32;      // [m + n] bin coordinates: the m row coordinates (f1 slabs), then the n column ones (f2 slabs)
    const double* X64;     // the same in FP64
    const float2* csum2;   // [m + n] C(x) = sum_y (X_x - X_y)^2 within each axis, as pairs
    struct CycleK* cyc;    // Prop. 3 constants of the current cycle
    HotCtl* ctl;
};

// ---- geometry of an m x n instance.  f1 slabs s < n (one per column j) are
// m x m (rows k, columns i); f2 slabs s = n + k (one per row k) are n x n
// (rows j, columns l).  Per-slab arrays are packed slab after slab; for
// m = n = S every offset below is the square layout's s S^2, s S, ...
__host__ __device__ inline int g_nslab(const HotInst& I) { return I.n + I.m; }
__host__ __device__ inline int g_side(const HotInst& I, int s) { return s < I.n ? I.m : I.n; }
__host__ __device__ inline int g_nb(const HotInst& I, int s) { return s < I.n ? I.nb1 : I.nb2; }
// A slab's rows are stored at a pitch of its side rounded up to a multiple of
// 4 (16 bytes in FP32), so that every row starts aligned for the vector loads
// of the sweeps; the pad columns hold zeros and take part in no sum.
__host__ __device__ inline int g_pitch(const HotInst& I, int s) { return s < I.n ? I.mp : I.np; }
// first flow variable of slab s (row r, column c at g_elem + r * g_pitch + c)
__host__ __device__ inline size_t g_elem(const HotInst& I, int s) {
    return s < I.n ? (size_t)s * I.m * I.mp : (size_t)I.n * I.m * I.mp + (size_t)(s - I.n) * I.n * I.np;
}
// entries of one state array: the slabs with their pad columns
__host__ __device__ inline size_t g_state_len(const HotInst& I) { return (size_t)I.m * I.n * ((size_t)I.mp + I.np); }
// first entry of slab s in arrays with one entry per slab row (or column)
__host__ __device__ inline size_t g_row(const HotInst& I, int s) {
    return s < I.n ? (size_t)s * I.m : (size_t)I.n * I.m + (size_t)(s - I.n) * I.n;
}
// first entry of (slab s, band) in the column-partial arrays [slab][band][column]
__host__ __device__ inline size_t g_colp(const HotInst& I, int s, int band) {
    return s < I.n ? ((size_t)s * I.nb1 + band) * I.m
                   : (size_t)I.n * I.nb1 * I.m + ((size_t)(s - I.n) * I.nb2 + band) * I.n;
}
__host__ __device__ inline int g_ntiles(const HotInst& I) { return I.n * I.nb1 + I.m * I.nb2; }
__host__ __device__ inline int g_tile(const HotInst& I, int s, int band) {
    return s < I.n ? s * I.nb1 + band : I.n * I.nb1 + (s - I.n) * I.nb2 + band;
}
__host__ __device__ inline void g_tile_slab(const HotInst& I, int t, int& s, int& band) {
    if (t < I.n * I.nb1) {
        s = t / I.nb1;
        band = t - s * I.nb1;
    } else {
        const int q = t - I.n * I.nb1;
        s = I.n + q / I.nb2;
        band = q - (s - I.n) * I.nb2;
    }
}
// first bin coordinate of slab s's half (row coordinates for f1, column for f2)
__host__ __device__ inline int g_xbase(const HotInst& I, int s) { return s < I.n ? 0 : I.m; }
// stride of the four instance-wide Prop. 3 vectors (indexed by j < n or k < m)
__host__ __device__ inline int g_L(const HotInst& I) { return I.m > I.n ? I.m : I.n; }

// Work tables of one batch, in device memory.  pre_* are prefix sums over the
// instances of the number of work items each kernel family handles.
struct WorkDev {
    int ninst;
    int alternate;         // the sweeps' state exceeds L2: odd iterations take the tiles in reverse
    HotInst* inst;         // [ninst]
    int* pre_tile;         // sweep / restart tiles: n nb1 + m nb2 per instance
    int* pre_slab;         // k_alpha: m + n slabs per instance
    int* pre_vec;          // k_vec: 2(m + n) per instance (one warp each); k_vec32: vec32_items(m, n) CTA items
    int* pre_k1;           // k_kkt1: n_k1 per instance
    int* pre_achunk;       // k_alpha32: n_achunk per instance
    int* n_running;        // instances still running
    int* st_out;           // [ninst] status of each instance after its last check
};

// Host-side launch helpers (hot_kernels.cu).
struct LaunchDims {
    // persistent grids: SM count x resident CTAs per SM of each kernel, so
    // that every CTA of a grid-stride loop is resident from the start
    int grid_tile;         // sweep
    int grid_tile_chk;     // sweep of check iterations
    int grid_rst;          // restart passes
    int grid_slab;
    int grid_alpha;        // k_alpha32 (FP32 mode)
    int grid_vec;
    int grid_vec1;         // k_vec32 of a single-instance batch (it also forms the stage)
    int grid_k1;
    int grid_inst;
};

// launches of one iteration: FP64 k_vec, k_marg, k_alpha, k_sweep64; FP32
// k_vec32, k_stage32 (batches of several instances only), k_alpha32, k_sweep32
inline int launches_per_iteration(int fp64, bool single) { return fp64 ? 4 : (single ? 3 : 4); }
inline int launches_per_block(int fp64, int K, bool single) { return K * launches_per_iteration(fp64, single); }
constexpr int kLaunchesBlockEnd = 8;       // k_kkt1, k_check, 3 x k_restart, k_restart_sigma, k_anchor, k_block_end
// work items of k_vec32 per instance: T1 (n outputs) and T2 (m outputs) in
// items of 8, P1 (m columns over n rows) and P2 (n columns over m rows) in items
// of 32 columns x 64 rows (one partial per 64-row block)
__host__ __device__ inline int vec32_items_dev(int m, int n) {
    return (n + 7) / 8 + (m + 7) / 8 + ((m + 31) / 32) * ((n + 63) / 64) + ((n + 31) / 32) * ((m + 63) / 64);
}
inline int vec32_items(int m, int n) { return vec32_items_dev(m, n); }
// float2 entries of vec2: T1, T2, then the (n + 63)/64 partials of P1 and the
// (m + 63)/64 partials of P2, then one row of per-item totals of the T1 and T2
// items ((n + 7)/8 + (m + 7)/8 <= max(m, n) entries), each a row of max(m, n)
inline size_t vec2_entries(int m, int n) {
    const int L = m > n ? m : n;
    return (size_t)(3 + (n + 63) / 64 + (m + 63) / 64) * L;
}
void launch_solve_kernels(const WorkDev* w, const LaunchDims& ld, int fp64, int j, bool check, bool single,
                          cudaStream_t st);
// pad: some instance of the batch has a side that is not a multiple of 4
void launch_sweep(const WorkDev* w, const LaunchDims& ld, int fp64, int j, bool check, bool pad, cudaStream_t st);
void launch_block_end(const WorkDev* w, const LaunchDims& ld, int fp64, int K, double a1, double a2, double a3,
                      cudaStream_t st);
LaunchDims make_launch_dims(int device, int fp64);
// resident CTAs of the (non-check) sweep on the current device
int sweep_grid(int fp64);
// u = -sigma0 c, d = 0, x_r = z_r = 0 and the FP64 sums of u for a new instance
// (the initial point w0 = 0: v0 = 0, y0 = 0).
void launch_init(const HotInst& I, double sigma0, cudaStream_t st);
cudaError_t kernels_init(int device);

}  // namespace hot
