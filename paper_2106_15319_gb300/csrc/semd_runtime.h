// Internal host-side declarations shared by the runtime and the server.
#pragma once
#include <string>

#include "semd_types.h"
#include "serial_emd.h"

namespace semd {

// One tile of TILE samples per CTA, TILE / kThreads consecutive samples per thread.
constexpr int kTile = 1024;
constexpr int kThreads = 128;

// Device workspace of a plan (or of a server slot pool): one allocation carved up.
struct Workspace {
    void *base = nullptr;
    size_t bytes = 0;
    int64_t cap_samples = 0, cap_tiles = 0, cap_rentries = 0;
    int cap_inst = 0, cap_iters = 0;
    size_t elem_size = 0;
    void *h0 = nullptr, *h1 = nullptr;
    double *r0 = nullptr, *r1 = nullptr;
    Inst *d_inst = nullptr;
    State *d_state = nullptr;
    int32_t *d_tile_inst = nullptr;
    TileExport *d_tex = nullptr;
    TileSolve *d_tsol = nullptr;
    TileAux *d_taux = nullptr;
    int64_t *d_rbase = nullptr;
    REntry *d_rent = nullptr;
    double *d_rA = nullptr, *d_rB = nullptr, *d_rC = nullptr, *d_rD = nullptr;
    double *d_rcp = nullptr, *d_rdp = nullptr, *d_rbp = nullptr, *d_rM = nullptr;
    int32_t *d_active = nullptr;
    double *d_beta = nullptr;
    int32_t *d_misc = nullptr;
    void *eemd_scratch = nullptr;
    // pinned host staging
    Inst *h_inst = nullptr;
    int32_t *h_tile_inst = nullptr;
    int64_t *h_rbase = nullptr;
    State *h_state = nullptr;
    void *h_misc = nullptr;
    cudaEvent_t staging_done = nullptr;

    semd_status allocate(int64_t samples, int insts, int64_t tiles, int64_t rentries, int iters,
                         size_t elem, int64_t eemd_elems, size_t budget, std::string &err);
    semd_status layout(int n, int64_t &ntiles, cudaStream_t s, std::string &err);
    void release();
};

int64_t serial_length(int64_t M, int64_t N, int64_t D);
bool geometry(const semd_params &p, int64_t rows, int64_t cols, int order, int64_t &M,
              int64_t &N, int64_t &D, std::string &err);
bool validate(const semd_params &p, std::string &err);
int max_iterations(const semd_params &p);

} // namespace semd

struct semd_plan_s {
    semd_params p;
    int64_t L = 0;
    semd::Workspace ws;
    std::string err;
    int last_ninst = 0, last_count = 0;
    void counts(int count, int *n_imfs, int *sifts) const;
};
