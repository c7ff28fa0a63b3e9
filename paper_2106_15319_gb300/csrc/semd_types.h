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
enum Stop : int32_t { STOP_FIXED = 0, STOP_SD = 1 };

// Per tile and envelope (0 = maxima, 1 = minima): what the interface solve needs of the
// tile's knots, after the tile has eliminated its interior knots.
// Values are in the pass kernel's working precision: double for FP64 plans, float (in
// the first half of each 8-byte slot) for FP32 ones; the interface solve widens them.
struct TileExport {
    int32_t n;     // knots of this kind in the tile
    int32_t t[4];  // instance positions of knots 0, 1, n-2, n-1
    int32_t pad;
    double y[4];   // their values
    double xa[3];  // M at knot 1   = xa[0] + xa[1] * M_0 + xa[2] * M_{n-1}  (n >= 3)
    double xb[3];  // M at knot n-2 = xb[0] + xb[1] * M_0 + xb[2] * M_{n-1}  (n >= 3)
};

// Per tile and envelope: the tile-boundary values solved by the interface solve.
// The FP64 solution, with a single-precision copy of every value for FP32 pass kernels.
struct TileSolve {
    double MF, ML;          // M at the tile's first and last knot
    int32_t tp, tn;         // outside bracket knots: last knot before the tile,
    double yp, Mp, yn, Mn;  // first knot after it (instance positions)
    float f[6];             // MF, ML, yp, Mp, yn, Mn in single precision
    int32_t pad[2];
};

// Working precision, like TileExport.
struct TileAux {
    double sd_num, sd_den;  // sum (h - h')^2, sum h^2 over the tile
    double h_first, h_last; // h[0] / h[L-1] of the new signal (first / last tile)
};

enum RKind : int32_t { RK_FIXED = 0, RK_FREE = 1, RK_F = 2, RK_L = 3, RK_FL = 4 };
struct REntry {
    int32_t t, tile, kind, pad;
    double y;
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
    TileExport *tex;        // 2 per tile
    TileSolve *tsol;        // 2 per tile
    TileAux *taux;          // 1 per tile
    REntry *rent;           // interface-solve scratch when it does not fit shared memory:
    double *rscr;           //   2 x rlen entries and 8 double arrays of 2 x rlen
    int64_t rlen;
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
    int32_t mode, hpar, rpar, imf_count, sift_count, nmax, nmin, pad;
    double sd;
    int32_t sifts[KMAX];
};

struct PassArgs {
    const Inst *inst;
    const State *state;
    const int32_t *tile_inst; // launch tile -> instance index
    Stats *stats;
};

struct ReduceArgs {
    const Inst *inst;
    State *state;
    const int32_t *inst_list; // block -> instance index (null: identity)
    int32_t *active;          // incremented once per instance still running
    int32_t K, stop, fixed_sifts, max_sifts;
    double sd_threshold;
    int32_t boundary, mirror_knots;
    int32_t single;       // 1: tile records hold floats (FP32 pass kernel)
    int32_t pad;
    int64_t smem_entries; // > 0: per-envelope scratch of this many entries in shared memory
};

// Shared memory of k_reduce for a per-envelope scratch of `entries` (skewed) entries.
__host__ __device__ inline size_t reduce_smem_bytes(int64_t entries)
{
    return 2 * (size_t)entries * (sizeof(REntry) + 8 * sizeof(double));
}

// Entries of the reduced system of an instance with nt tiles (per envelope).
__host__ __device__ constexpr int64_t reduce_entries(int nt) { return 2 * (int64_t)nt + 4; }
// Scratch length for n entries addressed through sk().
__host__ __device__ constexpr int64_t skew_len(int64_t n) { return n + n / 32 + 2; }

} // namespace semd
