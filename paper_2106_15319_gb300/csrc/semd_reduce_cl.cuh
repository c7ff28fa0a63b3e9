// Interface solve of long instances on a thread-block cluster.
//
// The interface system of an envelope (the reduced tridiagonal spline system of Sec. 2.1
// Step 2, partitioned by tiles: see semd_device.cuh) has about two rows per tile. One CTA
// holds it in shared memory up to about a thousand tiles; past that, the single-CTA
// kernel keeps its scratch in global memory and every phase waits on it. Here the system
// of one instance and envelope is spread over a cluster of CL CTAs (CL = 2..16) that
// exchange data through distributed shared memory:
//   - CTA c owns a contiguous range of tiles (counts, records, entries, the interface
//     values written back) and a contiguous range of RC = ceil(NR / CL) rows of the
//     system (trailing CTAs may own none); a tile's entries are stored into the shared
//     memory of the CTAs that own their rows.
//   - The rows are solved in four levels: every thread eliminates a run of its CTA's rows
//     (level 1); warp 0 of every CTA joins the runs into at most 32 groups (level 1.5);
//     warp 0 of CTA 0 joins all groups of the cluster into 32 lane blocks and solves the
//     32 block-end unknowns to FP64 accuracy (levels 1.75 and 2, the same 32-unknown core
//     as the single-CTA kernel); then each level is back-substituted.
// Every partition at every level has at least one row (balanced splits of what exists),
// so a run's successor is always the next run, in the same CTA or the next one.
// Natural spline ends only (not-a-knot plans use the single-CTA kernel).
#pragma once
#include <cooperative_groups.h>

#include "semd_device.cuh"

namespace semd {

namespace cgc = cooperative_groups;

constexpr int kClMax = 16;                  // CTAs per envelope at most (non-portable size)
constexpr int kClGroups = kClMax * 32;      // level-1.5 groups of a cluster at most
// Group arrays of CTA 0 are stored skewed (index j + j / 32), so that the lanes of the
// level-1.75 warp, which walk runs of consecutive groups at a fixed stride, hit distinct
// banks.
constexpr int kClGroupSlots = kClGroups + kClGroups / 32;
__host__ __device__ constexpr int gsk(int j) { return j + (j >> 5); }
constexpr size_t kClSmemOptin = 232448;     // shared memory per CTA an SM can give (227 KB)

// Counts of one CTA, published for the cluster-wide scan.
struct ClSum {
    double sdn, sdd; // SD sums of its tiles
    int U;           // reduced-system entries of its tiles
    int sn, so;      // knots of this envelope / the other one in its tiles
    int zs;          // zero crossings of the sifted signal in its tiles
    int done;        // the instance's state was DONE when this CTA read it
    int pad;
};

template <typename R>
struct ClShared {
    ClSum sum;
    // block-scan scratch
    double sd[kRedThreads / 32][2];
    int wsu[kRedThreads / 32], wsn[kRedThreads / 32][2], wzc[kRedThreads / 32];
    int next;
    // level 1: per run (thread) its elimination (10 values, run-major) and row count
    R lev[10][kRedThreads];
    int segq[kRedThreads];
    // level 1.5: per run of a group its elimination factors, then its end unknown
    R cp2[kRedThreads], dp2[kRedThreads], bp2[kRedThreads], zrun[kRedThreads];
    // CTA 0: every group's level-1.5 result (10 values, stored by the CTA that owns the
    // group), the level-1.75 factors per group and every group's end unknown
    R gg[10][kClGroupSlots];
    R cp3[kClGroupSlots], dp3[kClGroupSlots], bp3[kClGroupSlots], gz[kClGroupSlots];
};

// Bytes of ClShared at the start of the dynamic shared memory (16-byte multiple), and the
// whole dynamic shared memory of a CTA whose scratch holds `entries` entries.
template <typename R>
__host__ __device__ constexpr size_t cl_shared_bytes() { return (sizeof(ClShared<R>) + 15) & ~(size_t)15; }
template <typename R>
__host__ __device__ constexpr size_t cl_smem_bytes(int64_t entries)
{
    return cl_shared_bytes<R>() + red_env_bytes(entries, sizeof(R));
}

// Reduced-system entries one CTA stores for tiles per CTA T: its rows (at most 4 T + 1),
// the two halo rows, and slack.
__host__ __device__ constexpr int64_t cl_entries(int64_t T) { return 4 * T + 8; }

// Balanced split of n items into k non-empty parts (k <= n): part i is [lo, hi).
__device__ __forceinline__ void bsplit(int n, int k, int i, int &lo, int &hi)
{
    lo = (int)(((int64_t)n * i) / k);
    hi = (int)(((int64_t)n * (i + 1)) / k);
}

// Row g of the global system: the CTA that owns it and its slot there (slot 0 and RC + 1
// are the halo rows before and after the CTA's rows).
struct ClRows {
    int NR, RC;
    __device__ __forceinline__ int owner(int g) const { return g / RC; }
    __device__ __forceinline__ int slot(int g) const { return g - (g / RC) * RC + 1; }
    __device__ __forceinline__ int first(int c) const { return min(c * RC, NR); }
    __device__ __forceinline__ int count(int c) const { return min(RC, max(NR - c * RC, 0)); }
};

// Scratch arrays of another CTA of the cluster (the same layout in every CTA).
template <typename R>
__device__ __forceinline__ RedScratch<R> cl_remote(const cgc::cluster_group &cl,
                                                   const RedScratch<R> &X, int rank)
{
    RedScratch<R> Y;
    Y.Ey = cl.map_shared_rank(X.Ey, rank);
    Y.A = cl.map_shared_rank(X.A, rank);
    Y.B = cl.map_shared_rank(X.B, rank);
    Y.C = cl.map_shared_rank(X.C, rank);
    Y.D = cl.map_shared_rank(X.D, rank);
    Y.MV = cl.map_shared_rank(X.MV, rank);
    Y.Et = cl.map_shared_rank(X.Et, rank);
    Y.Ek = cl.map_shared_rank(X.Ek, rank);
    Y.St = cl.map_shared_rank(X.St, rank);
    Y.To = X.To;
    Y.Tu = X.Tu;
    return Y;
}

// One entry of a tile record (its k-th, of u), stored at slot q of scratch Y; the same
// entries as the one-CTA kernel's put_entries. Record fields are picked with selects, so
// that the record stays in registers.
template <typename R>
__device__ __forceinline__ void cl_put_entry(const RedScratch<R> &Y, int q, const TileRec<R> &rc,
                                             int k)
{
    const int n = rc.n;
    auto tk = [&](int i) { return i == 0 ? rc.t[0] : i == 1 ? rc.t[1] : i == 2 ? rc.t[2] : rc.t[3]; };
    auto yk = [&](int i) { return i == 0 ? rc.y[0] : i == 1 ? rc.y[1] : i == 2 ? rc.y[2] : rc.y[3]; };
    if (n == 1) {
        Y.Et[q] = rc.t[0];
        Y.Ey[q] = rc.y[0];
        Y.Ek[q] = EK_FL;
    } else if (n <= kSparseKnots) {
        // knots in order: t[0], (t[1] if n >= 3), (t[2] if n == 4), t[3]
        const int src = k == 0 ? 0 : (k == n - 1 ? 3 : k);
        Y.Et[q] = tk(src);
        Y.Ey[q] = yk(src);
        Y.Ek[q] = k == 0 ? EK_F : (k == n - 1 ? EK_L : EK_FREE);
    } else {
        const bool f = k == 0;
        Y.Et[q] = f ? rc.t[0] : rc.t[3];
        Y.Ey[q] = f ? rc.y[0] : rc.y[3];
        Y.Ek[q] = f ? EK_FS : EK_LS;
        Y.St[q] = f ? rc.t[1] : rc.t[2];
        Y.A[q] = f ? rc.y[1] : rc.y[2];
        Y.B[q] = f ? rc.xa[0] : rc.xb[0];
        Y.C[q] = f ? rc.xa[1] : rc.xb[1];
        Y.D[q] = f ? rc.xa[2] : rc.xb[2];
    }
}

// Reduced-system rows of one instance and envelope on a cluster (see the file comment).
// Grid: 2 CL CTAs per instance (cluster c of the launch: instance c / 2, envelope c % 2).
template <typename R>
__global__ void __launch_bounds__(kRedThreads, 1) k_reduce_cl(ReduceArgs ra)
{
    cgc::cluster_group cl = cgc::this_cluster();
    const int CL = (int)cl.num_blocks();
    const int c = (int)cl.block_rank();
    // dynamic shared memory: the CTA's ClShared, then its scratch (ra.smem_entries entries)
    extern __shared__ __align__(16) unsigned char rsm[];
    ClShared<R> &S = *reinterpret_cast<ClShared<R> *>(rsm);
    const int pair = (int)(blockIdx.x / CL);
    const int e = pair & 1;
    const int ii = ra.inst_list ? ra.inst_list[pair >> 1] : (pair >> 1);
    const Inst &in = ra.inst[ii];
    const int nt = in.ntiles;
    if (nt < ra.cl_min_nt || nt > ra.cl_max_nt)
        return; // the one-CTA kernel's instance (the same for every CTA of the cluster)
    const TileRec<R> *texe = reinterpret_cast<const TileRec<R> *>(in.tex) + (int64_t)e * nt;
    const TileRec<R> *texo = reinterpret_cast<const TileRec<R> *>(in.tex) + (int64_t)(e ^ 1) * nt;
    TileSolve *tsol = in.tsol + (int64_t)e * nt;
    const TileAux *taux = in.taux;
    RedScratch<R> X;
    X.carve(rsm + cl_shared_bytes<R>(), ra.cl_entries);
    const int T = (nt + CL - 1) / CL; // tiles per CTA
    const int ta = min(c * T, nt), tb = min(ta + T, nt), ntc = tb - ta;
    pdl_wait();
    // the next kernel may start now: the pass this solve waited for is complete, so the
    // next pass can read that pass's signal before its own wait
    pdl_trigger();
    State *st = ra.state + ii;
    const int mode_now = st->mode;
    const int pm = st->pass_mode, psift = st->pass_sift, pimf = st->pass_imf;
    const int ppar = st->pass_par, pscount = st->pass_scount;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NW = kRedThreads / 32;
    const bool want_sd = ra.stop == STOP_SD, want_zc = ra.stop == STOP_SNUMBER;

    // ---- counts of this CTA's tiles. With at most two tiles per thread, the thread loads
    // the whole records of its chunk of tiles here and keeps them for its entries;
    // otherwise records are counted in a block stride, four in flight per thread at a
    // time, and loaded again for the entries.
    int sn = 0, so_ = 0, zs = 0;
    double a = 0.0, b = 0.0;
    constexpr int kKeep = 2;
    const bool keep = ntc <= kKeep * kRedThreads;
    const int CH = (ntc + kRedThreads - 1) / kRedThreads;
    TileRec<R> rk[kKeep];
    if (keep) {
#pragma unroll
        for (int k = 0; k < kKeep; ++k) {
            const int t = tid * CH + k;
            rk[k].n = 0;
            if (k < CH && t < ntc) {
                rk[k] = load_rec(texe + ta + t);
                so_ += texo[ta + t].n;
                if (want_sd) {
                    a += taux[ta + t].sd_num;
                    b += taux[ta + t].sd_den;
                }
                if (want_zc)
                    zs += taux[ta + t].nzc;
            }
        }
#pragma unroll
        for (int k = 0; k < kKeep; ++k) {
            const int t = tid * CH + k;
            if (k < CH && t < ntc) {
                X.Tu[t] = (unsigned char)(rk[k].n <= kSparseKnots ? rk[k].n : 2);
                sn += rk[k].n;
            }
        }
    }
    for (int t0 = ta; !keep && t0 < tb; t0 += 4 * kRedThreads) {
        int ne[4], no[4], nz[4];
        double sa[4], sb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = t0 + tid + k * kRedThreads;
            ne[k] = no[k] = nz[k] = 0;
            sa[k] = sb[k] = 0.0;
            if (t < tb) {
                ne[k] = texe[t].n;
                no[k] = texo[t].n;
                if (want_sd) {
                    sa[k] = taux[t].sd_num;
                    sb[k] = taux[t].sd_den;
                }
                if (want_zc)
                    nz[k] = taux[t].nzc;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = t0 + tid + k * kRedThreads;
            if (t < tb)
                X.Tu[t - ta] = (unsigned char)(ne[k] <= kSparseKnots ? ne[k] : 2);
            sn += ne[k];
            so_ += no[k];
            zs += nz[k];
            a += sa[k];
            b += sb[k];
        }
    }
    sn = warp_sum(sn);
    so_ = warp_sum(so_);
    zs = warp_sum(zs);
    if (want_sd) {
        a = warp_sum(a);
        b = warp_sum(b);
    }
    if (lane == 0) {
        S.wsn[warp][0] = sn;
        S.wsn[warp][1] = so_;
        S.wzc[warp] = zs;
        S.sd[warp][0] = a;
        S.sd[warp][1] = b;
    }
    __syncthreads();
    // entry offsets within the CTA: a contiguous chunk of tiles per thread, a block scan
    const int ca = min(tid * CH, ntc), cb = min(ca + CH, ntc);
    int su = 0;
    for (int t = ca; t < cb; ++t)
        su += X.Tu[t];
    int incl = su;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        S.wsu[warp] = incl;
    __syncthreads();
    int ubase = incl - su, Uc = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        ubase += w < warp ? S.wsu[w] : 0;
        Uc += S.wsu[w];
    }
    if (tid == 0) {
        ClSum q;
        q.U = Uc;
        q.sn = q.so = q.zs = 0;
        q.sdn = q.sdd = 0.0;
        for (int w = 0; w < NW; ++w) {
            q.sn += S.wsn[w][0];
            q.so += S.wsn[w][1];
            q.zs += S.wzc[w];
            q.sdn += S.sd[w][0];
            q.sdd += S.sd[w][1];
        }
        q.done = mode_now == MODE_DONE ? 1 : 0;
        q.pad = 0;
        S.sum = q;
    }
    cl.sync(); // (1) every CTA's counts are published

    // ---- cluster totals and this CTA's entry offset (every warp: lane r reads CTA r)
    ClSum cs{};
    if (lane < CL)
        cs = *cl.map_shared_rank(&S.sum, lane);
    const int Ebefore = warp_sum(lane < c ? cs.U : 0);
    const int U = warp_sum(cs.U);
    const int ntot = warp_sum(cs.sn), nother = warp_sum(cs.so);
    const int zs_all = warp_sum(cs.zs);
    double sdn = 0.0, sdd = 0.0;
    if (want_sd) { // in rank order, the same sums in every CTA
        for (int r = 0; r < CL; ++r) {
            sdn += __shfl_sync(FULLMASK, cs.sdn, r);
            sdd += __shfl_sync(FULLMASK, cs.sdd, r);
        }
    }
    const bool done = __shfl_sync(FULLMASK, cs.done, 0) != 0; // rank 0's reading, for all
    if (done) {
        cl.sync(); // (2) no CTA leaves while another may still read its counts
        return;
    }
    if (tid == 0) { // the same decision in every CTA; rank 0 of the maxima records it
        const PassSnap ps{pm, psift, pimf, ppar, pscount};
        S.next = stop_step<R>(ra, in, st, e == 0 && c == 0, e, ntot, nother, sdn, sdd, zs_all, ps);
    }
    // rows: [nl boundary rows][U tile entries][nr boundary rows]; CTA r owns rows
    // [r RC, (r + 1) RC) at slots 1..
    const int nl = ra.boundary == BND_MIRROR ? min(ra.mirror_knots, ntot) : 1;
    const int nr = nl;
    const int NR = nl + U + nr;
    const ClRows rows{NR, (NR + CL - 1) / CL};
    const int r0 = rows.first(c), n = rows.count(c);
    auto at = [&](auto *local, int g) { // element of row g's slot, wherever it lives
        const int o = rows.owner(g);
        return (o == c ? local : cl.map_shared_rank(local, o)) + rows.slot(g);
    };
    // first entry row of every tile of this CTA (its chunk's running offsets), then the
    // entries: records in a block stride, four in flight per thread, each entry stored
    // in the shared memory of the CTA that owns its row
    {
        int p = nl + Ebefore + ubase;
        for (int t = ca; t < cb; ++t) {
            X.To[t] = p;
            p += X.Tu[t];
        }
    }
    __syncthreads();
    if (keep) {
#pragma unroll
        for (int k = 0; k < kKeep; ++k) {
            const int t = tid * CH + k;
            if (k < CH && t < ntc) {
                const int u = X.Tu[t], p = X.To[t];
                for (int j = 0; j < u; ++j) {
                    const int g = p + j, o = rows.owner(g);
                    cl_put_entry(o == c ? X : cl_remote(cl, X, o), rows.slot(g), rk[k], j);
                }
            }
        }
    }
    for (int t0 = 0; !keep && t0 < ntc; t0 += 4 * kRedThreads) {
        TileRec<R> rb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = t0 + tid + k * kRedThreads;
            if (t < ntc && X.Tu[t] > 0)
                rb[k] = load_rec(texe + ta + t);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = t0 + tid + k * kRedThreads;
            if (t >= ntc)
                break;
            const int u = X.Tu[t], p = X.To[t];
            for (int j = 0; j < u; ++j) {
                const int g = p + j, o = rows.owner(g);
                cl_put_entry(o == c ? X : cl_remote(cl, X, o), rows.slot(g), rb[k], j);
            }
        }
    }
    const int nm = S.next;
    cl.sync(); // (2) every entry is in place
    if (nm != MODE_SIFT && nm != MODE_SIFT_COMMIT)
        return; // the same in every CTA; nothing reads another CTA's memory after (2)

    // ---- boundary rows (natural ends: mirrored knots, or the end samples), computed from
    // the signal's first two / last two knots by the CTA that owns them
    auto boundary = [&](int g, int &t, R &y, int &k) {
        if (ra.boundary == BND_MIRROR) {
            if (g < nl) {
                const int f = nl;
                if (nl == 2 && g == 0) { // the signal's second knot, reflected
                    int t1;
                    R y1;
                    if (*at(X.Ek, f) == EK_FS) {
                        t1 = *at(X.St, f);
                        y1 = *at(X.A, f);
                    } else {
                        t1 = *at(X.Et, f + 1);
                        y1 = *at(X.Ey, f + 1);
                    }
                    t = -t1;
                    y = y1;
                    k = EK_FIXED;
                } else { // its first knot, reflected
                    t = -*at(X.Et, f);
                    y = *at(X.Ey, f);
                    k = nl == 2 ? EK_FREE : EK_FIXED;
                }
            } else {
                const int l = nl + U - 1, Lm = (int)(2 * (in.L - 1));
                if (g == l + 1) { // its last knot, reflected
                    t = Lm - *at(X.Et, l);
                    y = *at(X.Ey, l);
                    k = nr == 2 ? EK_FREE : EK_FIXED;
                } else { // its second-to-last knot, reflected
                    int t2;
                    R y2;
                    if (*at(X.Ek, l) == EK_LS) {
                        t2 = *at(X.St, l);
                        y2 = *at(X.A, l);
                    } else {
                        t2 = *at(X.Et, l - 1);
                        y2 = *at(X.Ey, l - 1);
                    }
                    t = Lm - t2;
                    y = y2;
                    k = EK_FIXED;
                }
            }
        } else {
            t = g == 0 ? 0 : (int)(in.L - 1);
            y = g == 0 ? (R)taux[0].h_first : (R)taux[nt - 1].h_last;
            k = EK_FIXED;
        }
    };
    auto is_boundary = [&](int g) { return g < nl || g >= nl + U; };
    if (tid < 4) { // rows 0, 1 and NR - 2, NR - 1, where boundary rows are
        const int g = tid < 2 ? tid : NR - 4 + tid;
        if (g >= 0 && g < NR && is_boundary(g) && rows.owner(g) == c && (tid < 2 || g >= 2)) {
            int t, k;
            R y;
            boundary(g, t, y, k);
            const int q = rows.slot(g);
            X.Et[q] = t;
            X.Ey[q] = y;
            X.Ek[q] = k;
        }
    } else if (n > 0 && (tid == 32 || tid == 64)) {
        // the halo rows next to this CTA's range: their positions and values
        const int g = tid == 32 ? r0 - 1 : r0 + n, q = tid == 32 ? 0 : n + 1;
        if (g >= 0 && g < NR) {
            int t, k;
            R y;
            if (is_boundary(g)) {
                boundary(g, t, y, k);
            } else {
                t = *at(X.Et, g);
                y = *at(X.Ey, g);
            }
            X.Et[q] = t;
            X.Ey[q] = y;
        }
    }
    __syncthreads();
    // ---- rows of this CTA (natural ends), as in the single-CTA kernel
    for (int j = tid; j < n; j += kRedThreads) {
        const int p = j + 1;
        const int k = X.Ek[p];
        R ra_ = R(0), rb_ = R(1), rc_ = R(0), rd = R(0);
        if (k != EK_FIXED) {
            const int tc = X.Et[p];
            const R yc = X.Ey[p];
            int tl = X.Et[p - 1], tr = X.Et[p + 1];
            R yl = X.Ey[p - 1], yr = X.Ey[p + 1];
            R x0 = R(0), x1 = R(0), x2 = R(0);
            if (k == EK_FS || k == EK_LS) {
                x0 = X.B[p];
                x1 = X.C[p];
                x2 = X.D[p];
                if (k == EK_FS) {
                    tr = X.St[p];
                    yr = X.A[p];
                } else {
                    tl = X.St[p];
                    yl = X.A[p];
                }
            }
            const R hl = R(tc - tl), hr = R(tr - tc);
            const R d0 = R(6) * ((yr - yc) * rrcp(hr) - (yc - yl) * rrcp(hl));
            const R a_ = hl, b_ = R(2) * (hl + hr), c_ = hr;
            ra_ = a_;
            rb_ = b_;
            rc_ = c_;
            rd = d0;
            if (k == EK_FS) {
                rb_ = b_ + c_ * x1;
                rc_ = c_ * x2;
                rd = d0 - c_ * x0;
            } else if (k == EK_LS) {
                rb_ = b_ + a_ * x2;
                ra_ = a_ * x1;
                rd = d0 - a_ * x0;
            }
        }
        X.A[p] = ra_;
        X.B[p] = rb_;
        X.C[p] = rc_;
        X.D[p] = rd;
    }
    __syncthreads();

    // ---- level 1: S1 runs of this CTA's rows, one per thread
    const int S1 = min(kRedThreads, n);
    int rs = 0, re = 0;
    if (tid < S1) {
        bsplit(n, S1, tid, rs, re);
        const SegElim<R> g = seg_eliminate_rows<R>(X.A + 1, X.B + 1, X.C + 1, X.D + 1, rs, re);
        const R gv[10] = {g.alS, g.beS, g.gaS, g.alE, g.beE, g.gaE, g.al, g.bl, g.cl, g.dl};
#pragma unroll
        for (int k = 0; k < 10; ++k)
            S.lev[k][tid] = gv[k];
        S.segq[tid] = re - rs;
    }
    // groups per CTA (NG of CTA r = min(32, its rows)) and the first group of each
    auto groups_of = [&](int r) { return r < CL ? min(32, rows.count(r)) : 0; };
    int G0 = 0, NGT = 0; // this CTA's first group; groups of the cluster
    {
        const int ngr = groups_of(lane);
        NGT = warp_sum(ngr);
        G0 = warp_sum(lane < c ? ngr : 0);
    }
    const int NG = groups_of(c);
    cl.sync(); // (3) every CTA's runs (a CTA's last run couples to the next CTA's first)

    // ---- level 1.5 (warp 0): group l of this CTA joins runs [sa, sb) of it
    int sa = 0, sb = 0;
    if (warp == 0 && lane < NG)
        bsplit(S1, NG, lane, sa, sb);
    if (warp == 0 && n > 0) {
        const bool next_cta = c + 1 < CL && rows.count(c + 1) > 0;
        R nx[3] = {R(0), R(0), R(0)}; // the next CTA's first run: alS, beS, gaS
        if (next_cta) {
            ClShared<R> *Sn = cl.map_shared_rank(&S, c + 1);
            nx[0] = Sn->lev[0][0];
            nx[1] = Sn->lev[1][0];
            nx[2] = Sn->lev[2][0];
        }
        auto red_row = [&](int j, R &A, R &B, R &C, R &D) {
            SegElim<R> gj;
            gj.alE = S.lev[3][j];
            gj.beE = S.lev[4][j];
            gj.gaE = S.lev[5][j];
            gj.al = S.lev[6][j];
            gj.bl = S.lev[7][j];
            gj.cl = S.lev[8][j];
            gj.dl = S.lev[9][j];
            const bool inside = j + 1 < S1;
            const R nalS = inside ? S.lev[0][j + 1] : nx[0];
            const R nbeS = inside ? S.lev[1][j + 1] : nx[1];
            const R ngaS = inside ? S.lev[2][j + 1] : nx[2];
            reduced_row(gj, S.segq[j], inside || next_cta, nalS, nbeS, ngaS, A, B, C, D);
        };
        if (lane < NG) {
            SegElim<R> g2;
            R cprev = R(0), dprev = R(0), bprev = R(1);
            for (int j = sa; j < sb - 1; ++j) {
                R A, B, C, D;
                red_row(j, A, B, C, D);
                const R inv = rrcp(B - A * cprev);
                cprev = C * inv;
                dprev = (D - A * dprev) * inv;
                bprev = -A * bprev * inv;
                S.cp2[j] = cprev;
                S.dp2[j] = dprev;
                S.bp2[j] = bprev;
            }
            red_row(sb - 1, g2.al, g2.bl, g2.cl, g2.dl);
            if (sb - sa >= 2) {
                g2.alE = dprev;
                g2.beE = bprev;
                g2.gaE = -cprev;
                R xa = g2.alE, xb = g2.beE, xg = g2.gaE;
                for (int j = sb - 3; j >= sa; --j) {
                    const R cc = S.cp2[j];
                    xa = S.dp2[j] - cc * xa;
                    xb = S.bp2[j] - cc * xb;
                    xg = -cc * xg;
                }
                g2.alS = xa;
                g2.beS = xb;
                g2.gaS = xg;
            }
            // into CTA 0, which joins the groups of the whole cluster
            const R gv[10] = {g2.alS, g2.beS, g2.gaS, g2.alE, g2.beE, g2.gaE, g2.al, g2.bl, g2.cl, g2.dl};
            ClShared<R> *S0 = cl.map_shared_rank(&S, 0);
#pragma unroll
            for (int k = 0; k < 10; ++k)
                S0->gg[k][gsk(G0 + lane)] = gv[k];
        }
    }
    cl.sync(); // (4) every CTA's groups, in CTA 0

    // ---- levels 1.75 and 2 (CTA 0, warp 0): lane L joins groups [ja, jb) of the cluster;
    // the 32 lane-end unknowns are solved to FP64 accuracy; then every group's end unknown
    if (c == 0 && warp == 0) {
        const int NL = min(32, NGT);
        int ja = 0, jb = 0;
        if (lane < NL)
            bsplit(NGT, NL, lane, ja, jb);
        // reduced row of group j of the cluster (every group has at least one run)
        auto gred_row = [&](int j, R &A, R &B, R &C, R &D) {
            SegElim<R> gj;
            gj.alE = S.gg[3][gsk(j)];
            gj.beE = S.gg[4][gsk(j)];
            gj.gaE = S.gg[5][gsk(j)];
            gj.al = S.gg[6][gsk(j)];
            gj.bl = S.gg[7][gsk(j)];
            gj.cl = S.gg[8][gsk(j)];
            gj.dl = S.gg[9][gsk(j)];
            const bool hn = j + 1 < NGT;
            reduced_row(gj, 1, hn, hn ? S.gg[0][gsk(j + 1)] : R(0), hn ? S.gg[1][gsk(j + 1)] : R(0),
                        hn ? S.gg[2][gsk(j + 1)] : R(0), A, B, C, D);
        };
        SegElim<R> g3;
        if (lane < NL) {
            R cprev = R(0), dprev = R(0), bprev = R(1);
            for (int j = ja; j < jb - 1; ++j) {
                R A, B, C, D;
                gred_row(j, A, B, C, D);
                const R inv = rrcp(B - A * cprev);
                cprev = C * inv;
                dprev = (D - A * dprev) * inv;
                bprev = -A * bprev * inv;
                S.cp3[gsk(j)] = cprev;
                S.dp3[gsk(j)] = dprev;
                S.bp3[gsk(j)] = bprev;
            }
            gred_row(jb - 1, g3.al, g3.bl, g3.cl, g3.dl);
            if (jb - ja >= 2) {
                g3.alE = dprev;
                g3.beE = bprev;
                g3.gaE = -cprev;
                R xa = g3.alE, xb = g3.beE, xg = g3.gaE;
                for (int j = jb - 3; j >= ja; --j) {
                    const R cc = S.cp3[gsk(j)];
                    xa = S.dp3[gsk(j)] - cc * xa;
                    xb = S.bp3[gsk(j)] - cc * xb;
                    xg = -cc * xg;
                }
                g3.alS = xa;
                g3.beS = xb;
                g3.gaS = xg;
            }
        }
        const double Zd = level2_solve(g3, jb - ja, lane < NL - 1);
        const R z = (R)Zd;
        R Zp = __shfl_up_sync(FULLMASK, z, 1);
        if (lane == 0)
            Zp = R(0);
        if (lane < NL) {
            S.gz[gsk(jb - 1)] = z;
            R xn = z;
            for (int j = jb - 2; j >= ja; --j) {
                const R x = S.dp3[gsk(j)] + S.bp3[gsk(j)] * Zp - S.cp3[gsk(j)] * xn;
                S.gz[gsk(j)] = x;
                xn = x;
            }
        }
    }
    cl.sync(); // (5) every group's end unknown, in CTA 0

    // ---- back-substitution: runs of every group (warp 0), then rows of every run
    if (warp == 0 && lane < NG) {
        const R *gz = cl.map_shared_rank(S.gz, 0);
        const int J = G0 + lane;
        const R z = gz[gsk(J)], Zp = J > 0 ? gz[gsk(J - 1)] : R(0);
        S.zrun[sb - 1] = z;
        R xn = z;
        for (int j = sb - 2; j >= sa; --j) {
            const R x = S.dp2[j] + S.bp2[j] * Zp - S.cp2[j] * xn;
            S.zrun[j] = x;
            xn = x;
        }
    }
    __syncthreads();
    if (tid < S1) {
        // the unknown before the run: the previous run's end (for a CTA's first run, the
        // previous CTA's last group's end)
        const R Zp = tid > 0 ? S.zrun[tid - 1]
                             : (G0 > 0 ? cl.map_shared_rank(S.gz, 0)[gsk(G0 - 1)] : R(0));
        seg_backsub_rows<R>(X.A + 1, X.C + 1, X.D + 1, X.MV + 1, rs, re, Zp, S.zrun[tid]);
    }
    cl.sync(); // (6) every row's second derivative

    // ---- the interface values of this CTA's tiles (rows next to and of their entries)
    for (int t = tid; t < ntc; t += kRedThreads) {
        const int u = X.Tu[t], p = X.To[t];
        TileSolve *so = tsol + ta + t;
        const R yp = *at(X.Ey, p - 1), Mp = *at(X.MV, p - 1);
        const R yn = *at(X.Ey, p + u), Mn = *at(X.MV, p + u);
        const R MF = u >= 1 ? *at(X.MV, p) : R(0), ML = u >= 1 ? *at(X.MV, p + u - 1) : R(0);
        const R M1 = u >= 3 ? *at(X.MV, p + 1) : R(0), M2 = u >= 4 ? *at(X.MV, p + 2) : R(0);
        so->tp = *at(X.Et, p - 1);
        so->tn = *at(X.Et, p + u);
        if (sizeof(R) == 4) {
            *reinterpret_cast<float4 *>(&so->f[0]) =
                make_float4((float)MF, (float)ML, (float)yp, (float)Mp);
            *reinterpret_cast<float4 *>(&so->f[4]) =
                make_float4((float)yn, (float)Mn, (float)M1, (float)M2);
        } else {
            so->MF = (double)MF;
            so->ML = (double)ML;
            so->yp = (double)yp;
            so->Mp = (double)Mp;
            so->yn = (double)yn;
            so->Mn = (double)Mn;
            so->M1 = (double)M1;
            so->M2 = (double)M2;
        }
    }
    cl.sync(); // (7) no CTA leaves while another may still read its rows
}

} // namespace semd
