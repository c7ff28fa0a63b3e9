// Internal host-side declarations shared by the runtime and the server.
#pragma once
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "semd_types.h"
#include "serial_emd.h"

namespace semd {

// One tile of TILE samples per warp, TILE / 32 consecutive samples per lane, kPassWarps
// independent warps per CTA. Supported tiles: 128, 256, 512; the plan picks one.
constexpr int kTile = 256;
constexpr int kMinTile = 128;
constexpr int kMaxTile = 512;
constexpr int kPassWarps = 4;
// Largest dynamic shared-memory scratch of the interface solve; larger instances use
// global memory.
constexpr size_t kReduceSmemMax = 184 * 1024;

// A named NVTX range over a host scope (decompositions, CEEMDAN stages, autotuning, server
// rounds), so that a timeline profiler shows where the host enqueues which work. Without a
// profiler attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Device workspace of a plan: one allocation carved up, plus pinned host staging.
struct Workspace {
    void *base = nullptr;
    size_t bytes = 0;
    int tile = kTile;
    int pass_ctas = 0;    // CTAs per SM of the persistent pass grid (0: as many as fit)
    int pass_variant = 0; // register budget of the pass kernel, where it has two
    int64_t cap_samples = 0, cap_tiles = 0, cap_rentries = 0; // cap_rentries: doubles of interface scratch
    int64_t max_ntiles = 0, min_ntiles = 0; // tile counts of the batch's longest / shortest instance
    int cap_inst = 0, cap_iters = 0;
    size_t elem_size = 0;
    void *h0 = nullptr, *h1 = nullptr;
    double *r0 = nullptr, *r1 = nullptr;
    Inst *d_inst = nullptr;
    State *d_state = nullptr;
    int32_t *d_tile_inst = nullptr;
    void *d_tex = nullptr;
    TileSolve *d_tsol = nullptr;
    TileAux *d_taux = nullptr;
    uint2 *d_kmask = nullptr; // 32 per tile
    double *d_rscr = nullptr; // interface-solve scratch: 16 x rlen doubles per instance
    int32_t *d_active = nullptr;
    double *d_beta = nullptr;
    int32_t *d_misc = nullptr;
    Stats *d_stats = nullptr;
    void *eemd_scratch = nullptr;
    // CEEMDAN (ensemble plans): call arguments, stage state, noise mode counts, r_k
    CeArgs *d_ce = nullptr;
    CeState *d_cestate = nullptr;
    int32_t *d_cecount = nullptr;
    double *d_ce_r = nullptr;
    CePart *d_cepart = nullptr; // one per stage-test block
    // pinned host staging
    Inst *h_inst = nullptr;
    int32_t *h_tile_inst = nullptr;
    State *h_state = nullptr;
    void *h_misc = nullptr;
    Stats *h_stats = nullptr;
    CeArgs *h_ce = nullptr;
    CeState *h_cestate = nullptr;
    cudaEvent_t staging_done = nullptr;

    semd_status allocate(int64_t samples, int insts, int64_t tiles, int64_t rentries, int iters,
                         size_t elem, int64_t eemd_elems, size_t budget, std::string &err);
    semd_status layout(int n, int64_t &ntiles, cudaStream_t s, std::string &err);
    void release();
};

// Per-instance scratch length of the interface solve (entries per envelope), a multiple
// of 4 so that every array of the scratch (8- and 4-byte elements, two envelopes) stays
// naturally aligned.
constexpr int64_t reduce_len(int64_t ntiles) { return (reduce_entries(ntiles) + 3) & ~(int64_t)3; }

int64_t serial_length(int64_t M, int64_t N, int64_t D);
bool geometry(const semd_params &p, int64_t rows, int64_t cols, int order, int64_t &M,
              int64_t &N, int64_t &D, std::string &err);
bool validate(const semd_params &p, std::string &err);
int max_iterations(const semd_params &p);

// Kernel launches for other translation units (the kernels are instantiated once, in the
// runtime's). elem is the working precision's size: 4 (FP32-mixed) or 8 (FP64).
cudaError_t setup_kernel_attrs(size_t elem);
// ctas_per_sm > 0 caps the persistent pass grid at that many CTAs per SM.
void launch_pass_any(size_t elem, int tile, const PassArgs &pa, int64_t ntiles, cudaStream_t s,
                     int ctas_per_sm = 0);
void launch_reduce_any(size_t elem, const ReduceArgs &ra, int nblocks, cudaStream_t s);
void launch_serialize_any(size_t elem, const Inst *d_inst, const State *d_state,
                          const int32_t *tile_inst, int64_t ntiles, int tile, cudaStream_t s);
void launch_finalize_any(size_t elem, const Inst *d_inst, const State *d_state,
                         const int32_t *tile_inst, int64_t ntiles, int tile, int K,
                         cudaStream_t s);
ReduceArgs make_reduce_args(const semd_params &p, const Inst *d_inst, State *d_state,
                            const int32_t *inst_list, int32_t *active, size_t elem,
                            int64_t min_ntiles, int64_t max_ntiles);
void choose_pass_shape(const semd_params &p, int64_t L, int ninst, int &tile, int &ctas,
                       int &variant);
// CTAs of the pass kernel that fit on one SM (working-precision size elem, tile, variant).
int pass_ctas_per_sm_max(size_t elem, int tile, int variant);
// Every pass kernel comes in two variants: 0 stages the next tile in shared memory, 1 does
// not (smaller; for FP32 256-sample tiles also a larger register budget).
inline bool pass_has_variants(size_t, int) { return true; }
// The tuning table (semd_autotune.cu): the entry for this plan key, if any.
bool tune_lookup(const semd_params &p, int64_t L, int ninst, int &tile, int &ctas,
                 int &variant);
template <typename R>
semd_status decompose_impl(semd_plan_s &pl, int count, const semd_instance *insts,
                           const void *d_noise, int *n_imfs, cudaStream_t s,
                           int64_t imf_stride_all);

// Optional per-launch timing of the pass and reduce kernels (CUDA events on the
// launching stream), used by the benchmark's roofline figures.
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<std::pair<int, size_t>> rec; // (kind, index of the start event)
    size_t used = 0;
    void reset()
    {
        rec.clear();
        used = 0;
    }
    size_t begin(int kind, cudaStream_t s)
    {
        while (ev.size() < used + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess)
                return (size_t)-1;
            ev.push_back(e);
        }
        cudaEventRecord(ev[used], s);
        rec.push_back({kind, used});
        used += 2;
        return rec.size() - 1;
    }
    void end(size_t slot, cudaStream_t s)
    {
        if (slot != (size_t)-1)
            cudaEventRecord(ev[rec[slot].second + 1], s);
    }
    void totals(double ms[2], int64_t cnt[2]) const
    {
        ms[0] = ms[1] = 0.0;
        cnt[0] = cnt[1] = 0;
        for (auto &r : rec) {
            float t = 0.f;
            cudaEventSynchronize(ev[r.second + 1]);
            if (cudaEventElapsedTime(&t, ev[r.second], ev[r.second + 1]) == cudaSuccess) {
                ms[r.first] += t;
                cnt[r.first] += 1;
            }
        }
    }
    // Device time of each profiled launch of one kind, in launch order (waits for the
    // events); returns how many launches of that kind were recorded.
    int64_t times(int kind, float *ms, int64_t cap) const
    {
        int64_t n = 0;
        for (auto &r : rec) {
            if (r.first != kind)
                continue;
            if (ms && n < cap) {
                float t = 0.f;
                cudaEventSynchronize(ev[r.second + 1]);
                if (cudaEventElapsedTime(&t, ev[r.second], ev[r.second + 1]) != cudaSuccess)
                    t = -1.f;
                ms[n] = t;
            }
            ++n;
        }
        return n;
    }
    void destroy()
    {
        for (auto e : ev)
            cudaEventDestroy(e);
        ev.clear();
        reset();
    }
};

struct GraphKey {
    int ninst = 0;
    int64_t ntiles = 0;
    int ntiles0 = 0;
    int64_t max_ntiles = 0;
    int tile = 0;
    int pass_ctas = 0;
    int pass_variant = 0;
    uint64_t seed = 0;
    int64_t min_ntiles = 0;
    bool operator==(const GraphKey &o) const
    {
        return ninst == o.ninst && ntiles == o.ntiles && ntiles0 == o.ntiles0 &&
               max_ntiles == o.max_ntiles && tile == o.tile && pass_ctas == o.pass_ctas &&
               pass_variant == o.pass_variant && seed == o.seed && min_ntiles == o.min_ntiles;
    }
};

} // namespace semd

struct semd_plan_s {
    semd_params p;
    int64_t L = 0;
    semd::Workspace ws;
    std::string err;
    int last_ninst = 0, last_count = 0;
    // CUDA graph of the fixed-sift-count decomposition, replayed on the plan's stream
    bool graphs = true;
    cudaStream_t gstream = nullptr;
    cudaStream_t lstream = nullptr; // captures the body of a device-decided sifting loop
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    semd::GraphKey graph_key;
    int64_t graph_launches = 0;
    // the same for CEEMDAN calls
    cudaGraphExec_t ce_graph_exec = nullptr;
    semd::GraphKey ce_graph_key;
    int64_t ce_graph_launches = 0;
    bool last_ceemdan = false; // the last call was CEEMDAN (counts come from its state)
    uint64_t noise_seed = 0;   // EEMD noise drawn by the library when the caller passes none
    // statistics of the last decomposition
    semd::Profiler prof;
    int64_t stat_launches = 0;
    int stat_graph = 0;
    void counts(int count, int *n_imfs, int *sifts) const;
};
