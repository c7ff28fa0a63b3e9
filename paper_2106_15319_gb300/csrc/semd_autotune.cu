// Autotuner of the sifting pass kernel's launch shape (host code).
//
// The pass kernel has three free launch parameters: the tile (128, 256 or 512 samples per
// warp, which moves work between the per-tile eliminations and the interface system),
// its variant (0 stages each warp's next tile in shared memory, 1 is a smaller kernel
// without staging that latency-bound launches prefer), and how many CTAs per SM its
// persistent grid keeps resident (fewer CTAs leave each one a longer contiguous range of
// tiles and more cache per CTA). None
// changes what is computed beyond rounding. serial_emd_plan_autotune times the plan's own
// decomposition of a caller's input for every candidate shape, keeps the fastest on the
// plan and records it in a process-wide table keyed by what decides the best shape:
// precision,
// stop rule, ensemble or not, and the log2 buckets of the instance count and of the
// longest serialized length. Plans created later with the same key start from the
// table's entry. The table can be saved to and merged from a JSON file.
#include "semd_runtime.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

namespace semd {

namespace {

struct TuneKey {
    int precision, stop, ensemble, batch_log2, len_log2;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(precision, stop, ensemble, batch_log2, len_log2) <
               std::tie(o.precision, o.stop, o.ensemble, o.batch_log2, o.len_log2);
    }
};

struct TuneVal {
    int tile = kTile, ctas = 0, variant = 0;
    double ms = 0.0;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
thread_local std::string g_tune_err;

int ceil_log2(int64_t v)
{
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < v)
        ++b;
    return b;
}

TuneKey make_key(const semd_params &p, int64_t L, int ninst)
{
    return TuneKey{p.precision, p.stop, p.ensemble_trials > 1 ? 1 : 0, ceil_log2(ninst),
                   ceil_log2(L)};
}

bool valid_shape(int tile, int ctas, int variant)
{
    return (tile == 128 || tile == 256 || tile == 512) && ctas >= 0 && ctas <= 64 &&
           (variant == 0 || variant == 1);
}

// One decomposition of the tuning input, enqueued on s.
semd_status run_once(semd_plan_s &pl, int count, const semd_instance *inst, const void *d_noise,
                     cudaStream_t s)
{
    return pl.p.precision == SEMD_FP64 ? decompose_impl<double>(pl, count, inst, d_noise,
                                                                nullptr, s, 0)
                                       : decompose_impl<float>(pl, count, inst, d_noise, nullptr,
                                                               s, 0);
}

// Median device time of `repeats` decompositions with the plan's current shape (after one
// untimed call, which also captures the shape's graph).
semd_status time_shape(semd_plan_s &pl, int count, const semd_instance *inst,
                       const void *d_noise, int repeats, cudaStream_t s, cudaEvent_t a,
                       cudaEvent_t b, double &ms)
{
    semd_status st = run_once(pl, count, inst, d_noise, s);
    if (st != SEMD_OK)
        return st;
    std::vector<double> t;
    for (int r = 0; r < repeats; ++r) {
        if (cudaEventRecord(a, s) != cudaSuccess)
            return SEMD_ECUDA;
        st = run_once(pl, count, inst, d_noise, s);
        if (st != SEMD_OK)
            return st;
        float e = 0.f;
        if (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&e, a, b) != cudaSuccess) {
            pl.err = "event timing failed during autotuning";
            return SEMD_ECUDA;
        }
        t.push_back(e);
    }
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return SEMD_OK;
}

} // namespace

bool tune_lookup(const semd_params &p, int64_t L, int ninst, int &tile, int &ctas,
                 int &variant)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(make_key(p, L, ninst));
    if (it == g_tune.end())
        return false;
    tile = it->second.tile;
    ctas = it->second.ctas;
    variant = it->second.variant;
    return true;
}

} // namespace semd

using namespace semd;

extern "C" {

semd_status serial_emd_plan_autotune(semd_plan_t plan, int count, const semd_instance *inst,
                                     const void *d_noise, int repeats, semd_tune_result *out,
                                     void *stream)
{
    if (!plan)
        return SEMD_EINVAL;
    NvtxRange nvtx("serial_emd_plan_autotune");
    semd_plan_s &pl = *plan;
    const bool eemd = pl.p.ensemble_trials > 1;
    if (!inst || count < 1 || count > (eemd ? 1 : pl.ws.cap_inst)) {
        pl.err = "autotune: count must be in [1, max_batch] (1 for ensemble plans)";
        return SEMD_EINVAL;
    }
    if (repeats < 1 || repeats > 100) {
        pl.err = "autotune: repeats must be in [1, 100]";
        return SEMD_EINVAL;
    }
    int64_t Lmax = 0;
    for (int i = 0; i < count; ++i) {
        int64_t M, N, D;
        if (!inst[i].d_x || !inst[i].d_imfs) {
            pl.err = "autotune: null input or output pointer";
            return SEMD_EINVAL;
        }
        if (!geometry(pl.p, inst[i].rows, inst[i].cols, pl.p.order, M, N, D, pl.err))
            return SEMD_EINVAL;
        Lmax = std::max(Lmax, serial_length(M, N, D));
    }
    if (Lmax > pl.L) {
        pl.err = "autotune: an input is larger than the plan's shape";
        return SEMD_EBUDGET;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a)
            cudaEventDestroy(a);
        pl.err = "autotune: event creation failed";
        return SEMD_ECUDA;
    }
    const int tile0 = pl.ws.tile, ctas0 = pl.ws.pass_ctas, var0 = pl.ws.pass_variant;
    const bool prof0 = pl.prof.on;
    pl.prof.on = false;
    const size_t elem = pl.p.precision == SEMD_FP64 ? 8 : 4;
    semd_tune_result res{};
    TuneVal best;
    best.ms = -1.0;
    semd_status st = SEMD_OK;
    int tried = 0;
    for (int tile : {256, 128, 512}) {
        for (int var = 0; var < (pass_has_variants(elem, tile) ? 2 : 1) && st == SEMD_OK;
             ++var) {
            const int fit = pass_ctas_per_sm_max(elem, tile, var);
            std::vector<int> cand = {0};
            for (int c : {1, 2, 3, 4, 6, 8})
                if (c < fit)
                    cand.push_back(c);
            for (int c : cand) {
                pl.ws.tile = tile;
                pl.ws.pass_ctas = c;
                pl.ws.pass_variant = var;
                double ms = 0.0;
                st = time_shape(pl, count, inst, d_noise, repeats, s, a, b, ms);
                if (st != SEMD_OK)
                    break;
                ++tried;
                if (tile == kTile && c == 0 && var == 0)
                    res.ms_default = ms;
                if (best.ms < 0.0 || ms < best.ms) {
                    best.tile = tile;
                    best.ctas = c;
                    best.variant = var;
                    best.ms = ms;
                }
            }
        }
        if (st != SEMD_OK)
            break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    pl.prof.on = prof0;
    if (st != SEMD_OK) {
        pl.ws.tile = tile0;
        pl.ws.pass_ctas = ctas0;
        pl.ws.pass_variant = var0;
        return st;
    }
    pl.ws.tile = best.tile;
    pl.ws.pass_ctas = best.ctas;
    pl.ws.pass_variant = best.variant;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[make_key(pl.p, Lmax, eemd ? pl.p.ensemble_trials : count)] = best;
    }
    res.tile = best.tile;
    res.ctas_per_sm = best.ctas;
    res.variant = best.variant;
    res.ms = best.ms;
    res.candidates = tried;
    if (out)
        *out = res;
    return SEMD_OK;
}

semd_status serial_emd_tune_lookup(const semd_params *params, int64_t L, int ninst, int *tile,
                                   int *ctas_per_sm, int *variant)
{
    if (!params || !tile || !ctas_per_sm || !variant || L < 1 || ninst < 1)
        return SEMD_EINVAL;
    int t = kTile, c = 0, v = 0;
    if (!tune_lookup(*params, L, ninst, t, c, v))
        return SEMD_PENDING;
    *tile = t;
    *ctas_per_sm = c;
    *variant = v;
    return SEMD_OK;
}

void serial_emd_tune_clear(void)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune.clear();
}

semd_status serial_emd_tune_save(const char *path)
{
    if (!path)
        return SEMD_EINVAL;
    std::string txt = "{\n  \"format\": \"serial_emd tuning table 1\",\n  \"entries\": [";
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        bool first = true;
        for (const auto &kv : g_tune) {
            char line[320];
            std::snprintf(line, sizeof line,
                          "%s\n    {\"precision\": %d, \"stop\": %d, \"ensemble\": %d, "
                          "\"batch_log2\": %d, \"len_log2\": %d, \"tile\": %d, "
                          "\"ctas_per_sm\": %d, \"variant\": %d, \"ms\": %.6f}",
                          first ? "" : ",", kv.first.precision, kv.first.stop,
                          kv.first.ensemble, kv.first.batch_log2, kv.first.len_log2,
                          kv.second.tile, kv.second.ctas, kv.second.variant, kv.second.ms);
            txt += line;
            first = false;
        }
    }
    txt += "\n  ]\n}\n";
    FILE *f = std::fopen(path, "wb");
    if (!f) {
        g_tune_err = std::string("cannot write ") + path;
        return SEMD_EINVAL;
    }
    const bool ok = std::fwrite(txt.data(), 1, txt.size(), f) == txt.size();
    if (std::fclose(f) != 0 || !ok) {
        g_tune_err = std::string("write failed: ") + path;
        return SEMD_EINVAL;
    }
    return SEMD_OK;
}

// Reads the entries of a file written by serial_emd_tune_save: every {...} object after
// "entries" is a flat set of "name": integer-or-number pairs. Objects that lack a field or
// hold an invalid shape are skipped; a file without an "entries" list is an error.
semd_status serial_emd_tune_load(const char *path)
{
    if (!path)
        return SEMD_EINVAL;
    FILE *f = std::fopen(path, "rb");
    if (!f) {
        g_tune_err = std::string("cannot read ") + path;
        return SEMD_EINVAL;
    }
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0)
        txt.append(buf, n);
    std::fclose(f);
    size_t pos = txt.find("\"entries\"");
    if (pos == std::string::npos || txt.find('[', pos) == std::string::npos) {
        g_tune_err = std::string("no \"entries\" list in ") + path;
        return SEMD_EINVAL;
    }
    pos = txt.find('[', pos) + 1;
    const size_t end = txt.find(']', pos);
    std::vector<std::pair<TuneKey, TuneVal>> got;
    while (pos < end) {
        const size_t ob = txt.find('{', pos);
        if (ob == std::string::npos || ob > end)
            break;
        const size_t cb = txt.find('}', ob);
        if (cb == std::string::npos || cb > end)
            break;
        const std::string obj = txt.substr(ob + 1, cb - ob - 1);
        pos = cb + 1;
        std::map<std::string, double> fld;
        size_t q = 0;
        while (true) {
            const size_t k0 = obj.find('"', q);
            if (k0 == std::string::npos)
                break;
            const size_t k1 = obj.find('"', k0 + 1);
            const size_t col = k1 == std::string::npos ? k1 : obj.find(':', k1);
            if (col == std::string::npos)
                break;
            const char *v0 = obj.c_str() + col + 1;
            char *v1 = nullptr;
            const double v = std::strtod(v0, &v1);
            if (v1 != v0)
                fld[obj.substr(k0 + 1, k1 - k0 - 1)] = v;
            q = (size_t)(v1 - obj.c_str());
            if (v1 == v0)
                q = col + 1;
        }
        static const char *need[] = {"precision", "stop", "ensemble", "batch_log2",
                                     "len_log2", "tile", "ctas_per_sm"};
        bool ok = true;
        for (const char *nm : need)
            ok = ok && fld.count(nm) && std::fabs(fld[nm]) < 1e6 &&
                 fld[nm] == std::floor(fld[nm]);
        if (!ok)
            continue;
        TuneKey k{(int)fld["precision"], (int)fld["stop"], (int)fld["ensemble"],
                  (int)fld["batch_log2"], (int)fld["len_log2"]};
        TuneVal v;
        v.tile = (int)fld["tile"];
        v.ctas = (int)fld["ctas_per_sm"];
        v.variant = fld.count("variant") ? (int)fld["variant"] : 0;
        v.ms = fld.count("ms") ? fld["ms"] : 0.0;
        if (!valid_shape(v.tile, v.ctas, v.variant) ||
            (fld.count("variant") && fld["variant"] != std::floor(fld["variant"])))
            continue;
        got.push_back({k, v});
    }
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto &kv : got)
        g_tune[kv.first] = kv.second;
    return SEMD_OK;
}

const char *serial_emd_tune_last_error(void) { return g_tune_err.c_str(); }

} // extern "C"
