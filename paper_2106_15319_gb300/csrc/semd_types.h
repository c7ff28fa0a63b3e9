// Data layout shared by the host runtime and the kernels of the GB300 Serial-EMD library
// (instances, per-instance state, per-tile records of the partitioned spline solve).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace semd {

constexpr int KMAX = 32;
constexpr unsigned FULLMASK = 0xffffffffu;

enum Mode : int32_t {
    MODE_INIT = 0,        // h <- (working precision) r; export h
    MODE_SIFT = 1,        // h <- sift(h); export
    MODE_SIFT_COMMIT = 2, // c <- sift(h); commit c; h <- r_new; export
    MODE_COMMIT = 3,      // c <- h; commit c; h <- r_new; export
    MODE_DONE = 4
};

enum Boundary : int32_t { BND_MIRROR = 0, BND_ENDPOINTS = 1 };
enum SplineEnd : int32_t { SPLINE_NATURAL = 0, SPLINE_NOT_A_KNOT = 1 };
enum Stop : int32_t { STOP_FIXED = 0, STOP_SD = 1, STOP_SNUMBER = 2 };

// Per tile and envelope (0 = maxima, 1 = minima): what the interface solve needs of the
// tile's knots, after the tile has eliminated its interior knots, in the pass kernel's
// working precision R (64 bytes for FP32, 112 for FP64; read with 16-byte loads).
template <typename R>
struct __align__(16) TileRec {
    int32_t n;    // knots of this kind in the tile
    int32_t t[4]; // instance positions of knots 0, 1, n-2, n-1
    R y[4];       // their values
    R xa[3];      // M at knot 1   = xa[0] + xa[1] * M_0 + xa[2] * M_{n-1}  (n >= 3)
    R xb[3];      // M at knot n-2 = xb[0] + xb[1] * M_0 + xb[2] * M_{n-1}  (n >= 3)
};
// Bytes of one record in a plan of element size `elem`.
__host__ __device__ constexpr size_t tile_rec_bytes(size_t elem)
{
    return elem == 4 ? sizeof(TileRec<float>) : sizeof(TileRec<double>);
}

// Per tile and envelope: the tile-boundary values solved by the interface solve. FP32
// plans fill the single-precision values (read by the FP32 pass kernel), FP64 plans the
// double ones.
struct __align__(16) TileSolve {
    float f[8];             // MF, ML, yp, Mp, yn, Mn, M1, M2 in single precision
    int32_t tp, tn;         // outside bracket knots: last knot before the tile, first knot
    int32_t pad[2];         // after it (instance positions)
    double MF, ML;          // M at the tile's first and last knot
    double yp, Mp, yn, Mn;  // values and M at the bracket knots
    double M1, M2;          // M at knots 1 and 2 (envelopes with at most 4 knots)
};

// Working precision, like TileExport.
struct TileAux {
    double sd_num, sd_den;  // sum (h - h')^2, sum h^2 over the tile
    double h_first, h_last; // h[0] / h[L-1] of the new signal (first / last tile)
    int32_t nzc;            // zero crossings of the sifted signal: pairs (k, k+1) with
    int32_t pad;            //   k + 1 in the tile and a sign change (S-number rule)
};

// Read-only description of one instance (one serialized signal) and its buffers. Every
// buffer is the instance's own, so instances can join and leave a batch between passes.
struct Inst {
    int64_t L;              // serialized length, Sec. 3.2: MN + DN - D
    int64_t M, N, D;        // signal length, number of signals, transition length
    int32_t tile0;          // first tile of the instance in the current launch
    int32_t ntiles;         // ceil(L / tile)
    int32_t order;          // 0: signal i is row i of the input, 1: column i
    int32_t imf_serialized; // 1: IMFs are written in serialized order (EEMD trials)
    void *h[2];             // working-precision signal, ping-pong (L elements each)
    double *r[2];           // FP64 residue, ping-pong (L elements each)
    void *tex;              // TileRec<R>, 2 per tile
    TileSolve *tsol;        // 2 per tile
    TileAux *taux;          // 1 per tile
    uint2 *kmask;           // 32 per tile: per lane, the extremum masks and ranks of the
                            //   signal the last pass wrote (read by the next sift)
    double *rscr;           // interface-solve scratch when it does not fit shared memory:
    int64_t rlen;           //   rlen entries per envelope, rscr_env_doubles(rlen) each
    const void *x;          // input (rows x cols, row-major), or null
    void *imf;              // IMF output base
    double *res;            // residue output (input shape), or null
    int64_t imf_stride;     // elements between IMF slots
    const void *noise;      // EEMD (instance 0): trials x L noise realizations
    void *avg_imf;          // EEMD (instance 0): averaged IMF output
    double *avg_res;        // EEMD (instance 0): averaged residue output, or null
};

// Device counters of one decomposition (summed by the pass kernel, one atomic per CTA).
struct Stats {
    unsigned long long sample_sifts; // serialized samples times sifts
    unsigned long long pass_bytes;   // algorithmic HBM bytes of the pass kernel
};

// Mutable per-instance state of the sifting state machine.
struct State {
    int32_t mode, hpar, rpar, imf_count, sift_count, nmax, nmin;
    int32_t scount; // S-number rule: consecutive sifts that met the count condition
    double sd;
    int32_t sifts[KMAX];
    // written by the pass kernel (the instance's first tile): the mode, sift and IMF
    // counts the pass ran with, so that both interface-solve CTAs of an instance read
    // the same inputs while one of them updates the fields above
    int32_t pass_mode, pass_sift, pass_imf, pass_par; // pass_par: hpar | rpar << 1
    int32_t pass_scount, pad;
};

struct PassArgs {
    const Inst *inst;
    State *state;
    const int32_t *tile_inst; // launch tile -> instance index
    int64_t ntiles;           // tiles in the launch
    int32_t need_sd;          // 1: accumulate the SD sums (SD stop rule, single-sift calls)
    int32_t need_zc;          // 1: count the sifted signal's zero crossings (S-number rule)
};

struct ReduceArgs {
    const Inst *inst;
    State *state;
    const int32_t *inst_list; // block -> instance index (null: identity)
    int32_t *active;          // incremented once per instance still running
    Stats *stats;             // per-decomposition counters, or null
    int32_t K, stop, fixed_sifts, max_sifts;
    double sd_threshold;
    int32_t boundary, mirror_knots;
    int32_t single;       // 1: tile records hold floats (FP32 pass kernel)
    int32_t s_number;     // S of the S-number rule
    int64_t smem_entries; // > 0: per-envelope scratch of this many entries in shared memory
    int32_t spline_end;   // SPLINE_NATURAL or SPLINE_NOT_A_KNOT
    // Instances of cl_min_nt..cl_max_nt tiles are solved by the cluster kernel (cl CTAs per
    // envelope, cl_entries entries of scratch per CTA), all others by the one-CTA kernel;
    // cl = 0: the one-CTA kernel for every instance. The choice depends on the instance's
    // tile count alone, so an instance's results do not depend on its batch.
    int32_t cl;
    int64_t cl_entries;
    int32_t cl_min_nt, cl_max_nt;
    int32_t run_single; // host: some instance of the launch takes the one-CTA kernel
    int32_t run_cl;     // host: some instance of the launch takes the cluster kernel
};

// One CEEMDAN call (Sec. 2.2, Steps 1-4), in device memory so that a captured graph can be
// replayed with other buffers. The trials are the plan's instances: first the EMD of every
// noise realization (its modes E_1..E_{K-1} stay in the ensemble scratch), then per stage
// the first EMD mode of r_k + beta_k E_k(w^(m)) for every trial.
struct CeArgs {
    const void *x;        // input, rows x cols (plan precision)
    const void *noise;    // trials x L noise realizations w^(m) (plan precision)
    const void *E;        // ensemble scratch: trial m's mode k at E + (m * K + k) * slot
    void *modes;          // K x rows x cols output (plan precision)
    double *res;          // residue output (input shape), or null
    double *r;            // residue r_k of the current stage, serialized (L doubles)
    int32_t *ncount;      // modes of each noise realization (trials)
    int64_t M, N, D, L;   // geometry of the input (Sec. 3.2)
    int64_t slot;         // elements between two mode slots of the scratch
    int32_t order, trials, K, pad;
    double rel;           // beta_k = rel * std(r_k)
};
struct CeState {
    double beta;          // beta_k of the current stage
    int32_t done;         // 1: a residue failed the IMF-start test, later stages are empty
    int32_t n;            // modes produced
    double mean;          // mean of r_k (first pass of the stage test)
    uint32_t arrived[2];  // blocks of the two stage-test passes that have finished
};
// Per-block partial results of the stage test.
struct CePart {
    double s;             // sum of r (first pass) or of (r - mean)^2 (second pass)
    int32_t nmax, nmin;   // extrema of r_k in the block's samples (second pass)
};
// Samples per block of the stage-test passes.
constexpr int kCeTestSpan = 2048;

// Threads of the interface-solve kernel (one CTA per instance and envelope), and of its
// form for launches whose instances all have at most kRedThreadsTiny tiles.
constexpr int kRedThreads = 256;
constexpr int kRedThreadsTiny = 64;

// Scratch of k_reduce for one envelope of `entries` entries: six arrays in the working
// precision, four of 32-bit integers and one of bytes, rounded to 16 bytes.
__host__ __device__ constexpr size_t red_env_bytes(int64_t entries, size_t elem)
{
    return ((size_t)entries * (6 * elem + 17) + 15) & ~(size_t)15;
}
// Global-memory scratch of one envelope, in doubles (sized for either precision).
__host__ __device__ constexpr int64_t rscr_env_doubles(int64_t entries)
{
    return (int64_t)(red_env_bytes(entries, 8) / 8);
}
// Shared memory of one k_reduce CTA when its scratch lives there.
__host__ __device__ constexpr size_t reduce_smem_bytes(int64_t entries, size_t elem)
{
    return red_env_bytes(entries, elem);
}

// Entries of the reduced system of an instance with nt tiles (per envelope).
// Envelopes of a tile with at most this many knots export all of them (no elimination of
// an interior), so the interface solve yields every knot's second derivative.
constexpr int kSparseKnots = 4;
__host__ __device__ constexpr int64_t reduce_entries(int64_t nt) { return kSparseKnots * nt + 4; }

} // namespace semd
