// Device side of the GB300 Serial-EMD library: data layout, the warp-level
// partitioned tridiagonal solver, and the two kernels of one sifting pass.
//
// Method (Zhang et al., arXiv 2106.15319): serialize the input (Sec. 3.2), sift the
// 1D signal (Sec. 2.1 Steps 1-5: extrema, cubic-spline envelopes, mean, subtract,
// stop test), commit IMFs (Eq. 1) and de-serialize (Sec. 3.3).
//
// Pass structure. Every instance's serialized signal is cut into tiles of TILE
// samples; one CTA owns one tile. A pass reads the current signal h once and writes
// the next one once:
//   k_pass    (per tile)  - extrema of h (Step 1), spline second derivatives of the
//                           tile's knots given the tile-boundary values solved by the
//                           previous k_reduce, envelope evaluation, mean and subtraction
//                           (Steps 2-4), SD partial sums, IMF commit (Step 5 / Eq. 1);
//                           then extrema of the new signal and elimination of the tile's
//                           interior knots (the per-chunk part of the partitioned
//                           spline solve), exported as a short record per tile.
//   k_reduce  (per instance) - assembles the reduced interface system (two unknowns
//                           per tile and envelope, plus the end knots), solves it in
//                           FP64, writes the tile-boundary values back, and runs the
//                           stop test / IMF state machine for the next pass.
// The knot lists never leave shared memory; only ~100 bytes per tile and envelope
// cross HBM besides the signal itself.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "semd_types.h"

namespace semd {

// Skewed index: lane l of a warp walking its own contiguous segment touches a
// different shared-memory bank than its neighbours.
__device__ __forceinline__ int sk(int j) { return j + (j >> 5); }

// Rounded arithmetic that the compiler may not contract into FMAs. Halo samples are
// computed twice (by the tile that owns them and by its neighbour); both copies must
// be bit-identical, so the evaluation uses explicit roundings.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
// Reciprocals: the hardware approximation in FP32 (about 2 ulp); in FP64 a float seed
// refined by two Newton steps (about 1 ulp), which avoids the long IEEE division
// sequence on the slow FP64 pipe. Both are deterministic, which is what the halo
// recomputation needs; neither is correctly rounded.
__device__ __forceinline__ float rrcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double rrcp(double a)
{
    double r = (double)__fdividef(1.0f, (float)a);
    double e = __fma_rn(-a, r, 1.0);
    r = __fma_rn(r, e, r);
    e = __fma_rn(-a, r, 1.0);
    return __fma_rn(r, e, r);
}
__device__ __forceinline__ float rdiv(float a, float b) { return __fmul_rn(a, rrcp(b)); }
__device__ __forceinline__ double rdiv(double a, double b) { return __dmul_rn(a, rrcp(b)); }

// ---------------------------------------------------------------------------------
// Warp-level partitioned tridiagonal solve.
//
// Unknowns x_0..x_{n-1}; row i: a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i, with the
// outside values x_{-1} = xl[col] and x_n = xr[col] given per right-hand-side column.
// Column 0 carries d; columns 1.. have d = 0 (they give the response to the outside
// values). Lane l owns rows [s, e); it eliminates rows s..e-2 with the Thomas
// algorithm in terms of x_{s-1} (last unknown of lane l-1) and x_{e-1} (its own last
// unknown Z_l), which leaves one reduced row per lane coupling Z_{l-1}, Z_l, Z_{l+1}.
// That 32-unknown system is solved by parallel cyclic reduction over shuffles, and
// (FULL) each lane back-substitutes its segment. Without FULL only the first and last
// unknowns are returned, per column. cp/dp/bp: per-row scratch (skewed index).
// The matrix is diagonally dominant (spline rows: b = 2(a + c)), so no pivoting.
template <typename R, int NCOL, bool FULL, class RowFn, class OutFn>
__device__ void warp_tridiag(int n, const RowFn &row, const R (&xl)[NCOL], const R (&xr)[NCOL],
                             R *cp, R *dp, R *bp, const OutFn &out, R (&first)[NCOL],
                             R (&last)[NCOL])
{
    const int lane = threadIdx.x & 31;
    const int Q = (n + 31) >> 5;
    const int s = min(lane * Q, n), e = min(s + Q, n), q = e - s;
    R alS = R(0), beS = R(0), gaS = R(1), alE = R(0), beE = R(1), gaE = R(0);
    R al = R(0), bl = R(1), cl = R(0), dl = R(0);
    if (q >= 2) {
        R cprev = R(0), dprev = R(0), bprev = R(0);
        for (int j = s; j <= e - 2; ++j) {
            R a, b, c, d;
            row(j, a, b, c, d);
            const R den = (j == s) ? b : b - a * cprev;
            const R inv = rrcp(den);
            const R cpj = c * inv;
            const R dpj = (d - a * dprev) * inv;
            const R bpj = ((j == s) ? -a : -a * bprev) * inv;
            cp[sk(j)] = cpj;
            dp[sk(j)] = dpj;
            bp[sk(j)] = bpj;
            cprev = cpj;
            dprev = dpj;
            bprev = bpj;
        }
        alE = dprev;
        beE = bprev;
        gaE = -cprev;
        R xa = alE, xb = beE, xg = gaE;
        for (int j = e - 3; j >= s; --j) {
            const R c = cp[sk(j)];
            xa = dp[sk(j)] - c * xa;
            xb = bp[sk(j)] - c * xb;
            xg = -c * xg;
        }
        alS = xa;
        beS = xb;
        gaS = xg;
    }
    if (q >= 1)
        row(e - 1, al, bl, cl, dl);
    const R nalS = __shfl_down_sync(FULLMASK, alS, 1);
    const R nbeS = __shfl_down_sync(FULLMASK, beS, 1);
    const R ngaS = __shfl_down_sync(FULLMASK, gaS, 1);
    const bool has_next = (q >= 1) && (e < n);
    R A = R(0), B = R(1), C = R(0), D[NCOL];
#pragma unroll
    for (int k = 0; k < NCOL; ++k)
        D[k] = R(0);
    if (q >= 1) {
        A = al * beE;
        B = bl + al * gaE + (has_next ? cl * nbeS : R(0));
        C = has_next ? cl * ngaS : R(0);
        D[0] = dl - al * alE - (has_next ? cl * nalS : R(0));
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NCOL; ++k)
                D[k] -= A * xl[k];
            A = R(0);
        }
        if (!has_next) {
#pragma unroll
            for (int k = 0; k < NCOL; ++k)
                D[k] -= cl * xr[k];
        }
    }
#pragma unroll
    for (int st = 1; st < 32; st <<= 1) {
        R Am = __shfl_up_sync(FULLMASK, A, st), Bm = __shfl_up_sync(FULLMASK, B, st);
        R Cm = __shfl_up_sync(FULLMASK, C, st);
        R Ap = __shfl_down_sync(FULLMASK, A, st), Bp = __shfl_down_sync(FULLMASK, B, st);
        R Cp = __shfl_down_sync(FULLMASK, C, st);
        R Dm[NCOL], Dp[NCOL];
#pragma unroll
        for (int k = 0; k < NCOL; ++k) {
            Dm[k] = __shfl_up_sync(FULLMASK, D[k], st);
            Dp[k] = __shfl_down_sync(FULLMASK, D[k], st);
        }
        if (lane < st) {
            Am = R(0);
            Bm = R(1);
            Cm = R(0);
#pragma unroll
            for (int k = 0; k < NCOL; ++k)
                Dm[k] = R(0);
        }
        if (lane + st >= 32) {
            Ap = R(0);
            Bp = R(1);
            Cp = R(0);
#pragma unroll
            for (int k = 0; k < NCOL; ++k)
                Dp[k] = R(0);
        }
        const R k1 = A * rrcp(Bm), k2 = C * rrcp(Bp);
        const R nA = -k1 * Am, nC = -k2 * Cp, nB = B - k1 * Cm - k2 * Ap;
#pragma unroll
        for (int k = 0; k < NCOL; ++k)
            D[k] = D[k] - k1 * Dm[k] - k2 * Dp[k];
        A = nA;
        B = nB;
        C = nC;
    }
    R Z[NCOL], Zp[NCOL];
    const R invB = rrcp(B);
#pragma unroll
    for (int k = 0; k < NCOL; ++k) {
        Z[k] = D[k] * invB;
        Zp[k] = __shfl_up_sync(FULLMASK, Z[k], 1);
        if (lane == 0)
            Zp[k] = xl[k];
    }
    if constexpr (FULL) {
        if (q >= 1) {
            out(e - 1, Z[0]);
            R xn = Z[0];
            for (int j = e - 2; j >= s; --j) {
                const R x = dp[sk(j)] + bp[sk(j)] * Zp[0] - cp[sk(j)] * xn;
                out(j, x);
                xn = x;
            }
        }
    } else {
        const int last_lane = (n - 1) / Q;
#pragma unroll
        for (int k = 0; k < NCOL; ++k) {
            const R f = (k == 0 ? alS : R(0)) + beS * xl[k] + gaS * Z[k];
            first[k] = __shfl_sync(FULLMASK, f, 0);
            last[k] = __shfl_sync(FULLMASK, Z[k], last_lane);
        }
    }
}

// Rows of the natural-spline system for the interior knots 1..m-2 of a tile
// (Sec. 2.1 Step 2, cubic spline): unknown i is knot i+1 with
//   h_l M_{j-1} + 2 (h_l + h_r) M_j + h_r M_{j+1} = 6 [(y_{j+1}-y_j)/h_r - (y_j-y_{j-1})/h_l].
template <typename R>
struct KnotRows {
    const int *kt; // tile-relative knot positions (skewed index)
    const R *sl;   // sl[j] = (y_{j+1} - y_j) / (t_{j+1} - t_j), skewed index
    __device__ void operator()(int i, R &a, R &b, R &c, R &d) const
    {
        const int tl = kt[sk(i)], tc = kt[sk(i + 1)], tr = kt[sk(i + 2)];
        const R hl = R(tc - tl), hr = R(tr - tc);
        a = hl;
        b = R(2) * (hl + hr);
        c = hr;
        d = R(6) * (sl[sk(i + 1)] - sl[sk(i)]);
    }
};

// Rows of the reduced interface system, read from global scratch.
struct ScratchRows {
    const double *A, *B, *C, *D;
    __device__ void operator()(int i, double &a, double &b, double &c, double &d) const
    {
        a = A[i];
        b = B[i];
        c = C[i];
        d = D[i];
    }
};

// One spline interval [tl, tr] with values (yl, yr) and second derivatives (Ml, Mr),
// in the local polynomial form e(u) = c0 + c1 u + c2 u^2 + c3 u^3, u = k - tl. This is
// the textbook interval formula expanded in powers of u.
template <typename R>
struct Interval {
    int tl, tr;
    R yr, c0, c1, c2, c3;
    __device__ void set(int tl_, R yl, R Ml, int tr_, R yr_, R Mr)
    {
        tl = tl_;
        tr = tr_;
        yr = yr_;
        const R h = R(tr_ - tl_);
        const R inv = rrcp(h);
        const R slope = rmul(rsub(yr_, yl), inv);
        c0 = yl;
        c1 = rsub(slope, rmul(rmul(h, radd(rmul(R(2), Ml), Mr)), R(1.0 / 6.0)));
        c2 = rmul(Ml, R(0.5));
        c3 = rmul(rmul(rsub(Mr, Ml), inv), R(1.0 / 6.0));
    }
    __device__ R eval(int k) const
    {
        if (k == tr)
            return yr;
        const R u = R(k - tl);
        return rfma(rfma(rfma(c3, u, c2), u, c1), u, c0);
    }
};

// ---------------------------------------------------------------------------------
// Shared memory of one tile pass. The signal itself lives in registers: lane l of warp
// w holds samples w*32*RW + 32*r + l, r < RW, so every warp-wide access to a row is 32
// consecutive samples (coalesced global traffic, conflict-free shared memory).
template <typename R, int TILE, int NT>
struct PassSmem {
    static constexpr int NW = NT / 32;                 // warps
    static constexpr int RW = TILE / NT;               // rows per warp = samples per lane
    static constexpr int KCAP = TILE / 2 + 2;          // knots of one kind in a tile
    static constexpr int SKN = KCAP + KCAP / 32 + 2;   // skewed length
    int kt[2][SKN];  // tile-relative knot positions
    R ky[2][SKN];    // knot values
    R kM[2][SKN];    // second derivatives at the knots
    R sl[2][SKN];    // knot-interval slopes (solver input)
    R cp[2][SKN], dp[2][SKN], bp[2][SKN]; // solver scratch, then interval coefficients c1..c3
    R edge_first[NW], edge_last[NW];
    uint32_t wtot[NW];
    double red[2][NW];
    int cnt[2];
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}

// De-serialized destination of serialized sample p (Sec. 3.3): returns false for
// transition samples, which the de-serialization drops.
__device__ __forceinline__ bool deser_index(int64_t p, int64_t M, int64_t N, int64_t D, int order,
                                            int64_t &dst)
{
    const int64_t i = p / (M + D), m = p - i * (M + D);
    if (m >= M)
        return false;
    dst = order == 0 ? i * M + m : m * N + i;
    return true;
}

__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }
__device__ __forceinline__ uint32_t lanemask_le() { return (2u << (threadIdx.x & 31)) - 1u; }

// Step 1 on the tile held in registers: extremum flags of v (maximum: h[k-1] < h[k] >=
// h[k+1]; minimum: h[k-1] > h[k] <= h[k+1]; never at the instance's end samples) as one
// ballot mask per row and envelope, their in-order ranks (wbase + pre + popc), and the
// compacted knot lists (position and value) in shared memory.
template <typename R, int TILE, int NT>
__device__ void detect_knots(PassSmem<R, TILE, NT> &S, const R (&v)[TILE / NT], R left_halo,
                             R right_halo, int cnt, int64_t ts, int64_t L,
                             uint32_t (&mx)[TILE / NT], uint32_t (&mn)[TILE / NT],
                             int (&wbase)[2], int (&pre)[2][TILE / NT])
{
    constexpr int RW = TILE / NT, NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        S.edge_first[w] = v[0];
    if (lane == 31)
        S.edge_last[w] = v[RW - 1];
    __syncthreads();
    const R prev_last = w > 0 ? S.edge_last[w - 1] : left_halo;
    const R next_first = w < NW - 1 ? S.edge_first[w + 1] : right_halo;
    int c0 = 0, c1 = 0;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int k = w * 32 * RW + 32 * r + lane;
        const R c = v[r];
        const R up = __shfl_up_sync(FULLMASK, c, 1);
        const R dn = __shfl_down_sync(FULLMASK, c, 1);
        const R pr = __shfl_sync(FULLMASK, v[r > 0 ? r - 1 : 0], 31);
        const R nx = __shfl_sync(FULLMASK, v[r < RW - 1 ? r + 1 : RW - 1], 0);
        const R left = lane > 0 ? up : (r > 0 ? pr : prev_last);
        const R right = lane < 31 ? dn : (r < RW - 1 ? nx : next_first);
        const int64_t g = ts + k;
        const bool valid = k < cnt && g >= 1 && g <= L - 2;
        mx[r] = __ballot_sync(FULLMASK, valid && left < c && c >= right);
        mn[r] = __ballot_sync(FULLMASK, valid && left > c && c <= right);
        pre[0][r] = c0;
        pre[1][r] = c1;
        c0 += __popc(mx[r]);
        c1 += __popc(mn[r]);
    }
    if (lane == 0)
        S.wtot[w] = (uint32_t)c0 | ((uint32_t)c1 << 16);
    __syncthreads();
    int b0 = 0, b1 = 0, t0 = 0, t1 = 0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {
        const uint32_t t = S.wtot[ww];
        if (ww < w) {
            b0 += (int)(t & 0xffffu);
            b1 += (int)(t >> 16);
        }
        t0 += (int)(t & 0xffffu);
        t1 += (int)(t >> 16);
    }
    wbase[0] = b0;
    wbase[1] = b1;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int k = w * 32 * RW + 32 * r + lane;
        if ((mx[r] >> lane) & 1u) {
            const int idx = b0 + pre[0][r] + __popc(mx[r] & lt);
            S.kt[0][sk(idx)] = k;
            S.ky[0][sk(idx)] = v[r];
        }
        if ((mn[r] >> lane) & 1u) {
            const int idx = b1 + pre[1][r] + __popc(mn[r] & lt);
            S.kt[1][sk(idx)] = k;
            S.ky[1][sk(idx)] = v[r];
        }
    }
    if (threadIdx.x == 0) {
        S.cnt[0] = t0;
        S.cnt[1] = t1;
    }
    __syncthreads();
}

// Slopes of the knot intervals of both envelopes, all threads in parallel (keeps the
// divisions out of the sequential elimination).
template <typename R, int TILE, int NT>
__device__ __forceinline__ void knot_slopes(PassSmem<R, TILE, NT> &S)
{
    const int n0 = max(S.cnt[0] - 1, 0), n1 = max(S.cnt[1] - 1, 0);
    for (int idx = threadIdx.x; idx < n0 + n1; idx += NT) {
        const int e = idx < n0 ? 0 : 1;
        const int j = idx < n0 ? idx : idx - n0;
        const int ta = S.kt[e][sk(j)], tb = S.kt[e][sk(j + 1)];
        S.sl[e][sk(j)] = rmul(rsub(S.ky[e][sk(j + 1)], S.ky[e][sk(j)]), rrcp(R(tb - ta)));
    }
}

// Interval q of envelope e spans (knot q-1, knot q), with knot -1 the bracket knot before
// the tile and knot m the one after it. Coefficients of the cubic in u = k - t_{q-1}:
// c0 = y_{q-1} (not stored), c1..c3 written over the solver scratch.
template <typename R, int TILE, int NT>
__device__ __forceinline__ void interval_coefs(PassSmem<R, TILE, NT> &S, const TileSolve &so0,
                                               const TileSolve &so1, int64_t ts)
{
    const int m0 = S.cnt[0], m1 = S.cnt[1];
    for (int idx = threadIdx.x; idx < m0 + m1 + 2; idx += NT) {
        const int e = idx <= m0 ? 0 : 1;
        const int q = idx <= m0 ? idx : idx - m0 - 1;
        const int m = e ? m1 : m0;
        const TileSolve &so = e ? so1 : so0;
        int tl, tr;
        R yl, Ml, yr, Mr;
        if (q == 0) {
            tl = (int)(so.tp - ts);
            yl = (R)so.yp;
            Ml = (R)so.Mp;
        } else {
            tl = S.kt[e][sk(q - 1)];
            yl = S.ky[e][sk(q - 1)];
            Ml = S.kM[e][sk(q - 1)];
        }
        if (q == m) {
            tr = (int)(so.tn - ts);
            yr = (R)so.yn;
            Mr = (R)so.Mn;
        } else {
            tr = S.kt[e][sk(q)];
            yr = S.ky[e][sk(q)];
            Mr = S.kM[e][sk(q)];
        }
        const R h = R(tr - tl);
        const R inv = rrcp(h);
        const R slope = rmul(rsub(yr, yl), inv);
        S.cp[e][sk(q)] = rsub(slope, rmul(rmul(h, radd(rmul(R(2), Ml), Mr)), R(1.0 / 6.0)));
        S.dp[e][sk(q)] = rmul(Ml, R(0.5));
        S.bp[e][sk(q)] = rmul(rmul(rsub(Mr, Ml), inv), R(1.0 / 6.0));
    }
}

// Envelope e at tile-relative sample k, which lies in interval q. The spline passes
// through its knots; at the bracket knot after the tile (only reachable when it sits
// on a sample, the ENDPOINTS rule's last sample) the knot value is returned exactly.
template <typename R, int TILE, int NT>
__device__ __forceinline__ R envelope_at(const PassSmem<R, TILE, NT> &S, int e, int q, int k,
                                         const TileSolve &so, int64_t ts)
{
    const int m = S.cnt[e];
    if (q == m && (int64_t)k == so.tn - ts)
        return (R)so.yn;
    const int tl = q > 0 ? S.kt[e][sk(q - 1)] : (int)(so.tp - ts);
    const R c0 = q > 0 ? S.ky[e][sk(q - 1)] : (R)so.yp;
    const R u = R(k - tl);
    return rfma(rfma(rfma(S.bp[e][sk(q)], u, S.dp[e][sk(q)]), u, S.cp[e][sk(q)]), u, c0);
}

// ---------------------------------------------------------------------------------
// One sifting pass over one tile. Grid: one CTA per tile of every instance.
template <typename R, int TILE, int NT>
__global__ void __launch_bounds__(NT) k_pass(PassArgs pa)
{
    constexpr int RW = TILE / NT, NW = NT / 32;
    static_assert(RW >= 1 && RW <= 32 && TILE % NT == 0 && NW >= 2, "tile split");
    extern __shared__ __align__(16) unsigned char smraw[];
    PassSmem<R, TILE, NT> &S = *reinterpret_cast<PassSmem<R, TILE, NT> *>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gt = blockIdx.x;
    const int ii = pa.tile_inst[gt];
    const State *stp = pa.state + ii;
    const int mode = stp->mode;
    if (mode == MODE_DONE)
        return;
    const int hpar = stp->hpar, rpar = stp->rpar, imfc = stp->imf_count;
    const Inst &in = pa.inst[ii];
    const int64_t L = in.L;
    const int64_t ts = (int64_t)(gt - in.tile0) * TILE;
    const int cnt = (int)min((int64_t)TILE, L - ts);
    const bool hasL = ts > 0, hasR = ts + cnt < L;
    const R *hsrc = (const R *)(hpar ? pa.h1 : pa.h0) + in.off + ts;
    R *hdst = (R *)(hpar ? pa.h0 : pa.h1) + in.off + ts;
    const double *rsrc = (rpar ? pa.r1 : pa.r0) + in.off + ts;
    double *rdst = (rpar ? pa.r0 : pa.r1) + in.off + ts;
    const bool sift = mode == MODE_SIFT || mode == MODE_SIFT_COMMIT;
    const bool commit = mode == MODE_SIFT_COMMIT || mode == MODE_COMMIT;
    const int kbase = warp * 32 * RW + lane;

    // current signal: samples k <= cnt (k == cnt is the right halo of a partial tile),
    // plus the halo of a full tile and the left halo, each in one register
    R v[RW];
    R hl = R(0), hr = R(0);
    if (mode != MODE_INIT) {
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int k = kbase + 32 * r;
            v[r] = (k < cnt || (k == cnt && hasR)) ? hsrc[k] : R(0);
        }
        if (tid == 0 && hasL)
            hl = hsrc[-1];
        if (tid == NT - 1 && hasR && cnt == TILE)
            hr = hsrc[TILE];
    }

    R hn[RW];
    R hnl = R(0), hnr = R(0);
    double sdn = 0.0, sdd = 0.0;
    if (sift) {
        uint32_t mx[RW], mn[RW];
        int wbase[2], pre[2][RW];
        detect_knots<R, TILE, NT>(S, v, hl, hr, cnt, ts, L, mx, mn, wbase, pre);
        const TileSolve so0 = pa.tsol[2 * (int64_t)gt], so1 = pa.tsol[2 * (int64_t)gt + 1];
        knot_slopes<R, TILE, NT>(S);
        __syncthreads();
        // Step 2: second derivatives at the tile's knots (one warp per envelope), with the
        // tile's first and last knot values from the interface solve
        if (warp < 2) {
            const int e = warp;
            const int m = S.cnt[e];
            const TileSolve &so = e ? so1 : so0;
            if (m >= 1 && lane == 0) {
                S.kM[e][sk(0)] = (R)so.MF;
                S.kM[e][sk(m - 1)] = (R)so.ML;
            }
            if (m >= 3) {
                const R xl[1] = {(R)so.MF}, xr[1] = {(R)so.ML};
                R f1[1], l1[1];
                R *kM = S.kM[e];
                warp_tridiag<R, 1, true>(
                    m - 2, KnotRows<R>{S.kt[e], S.sl[e]}, xl, xr, S.cp[e], S.dp[e], S.bp[e],
                    [kM](int i, R x) { kM[sk(i + 1)] = x; }, f1, l1);
            }
        }
        __syncthreads();
        interval_coefs<R, TILE, NT>(S, so0, so1, ts);
        __syncthreads();
        // Steps 2-4 at every sample: envelopes, mean, subtraction
        const uint32_t le = lanemask_le();
        R pn = R(0), pd = R(0);
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int k = kbase + 32 * r;
            const int q0 = wbase[0] + pre[0][r] + __popc(mx[r] & le);
            const int q1 = wbase[1] + pre[1][r] + __popc(mn[r] & le);
            if (k < cnt || (k == cnt && hasR)) {
                const R e0 = envelope_at(S, 0, q0, k, so0, ts);
                const R e1 = envelope_at(S, 1, q1, k, so1, ts);
                const R mean = rmul(radd(e0, e1), R(0.5));
                hn[r] = rsub(v[r], mean);
                if (k < cnt) {
                    pn += mean * mean;
                    pd += v[r] * v[r];
                }
            } else {
                hn[r] = R(0);
            }
        }
        sdn = (double)pn;
        sdd = (double)pd;
        if (tid == 0 && hasL) { // left halo: interval 0 of both envelopes
            const R mean = rmul(radd(envelope_at(S, 0, 0, -1, so0, ts),
                                     envelope_at(S, 1, 0, -1, so1, ts)), R(0.5));
            hnl = rsub(hl, mean);
        }
        if (tid == NT - 1 && hasR && cnt == TILE) { // right halo: the last interval
            const R mean = rmul(radd(envelope_at(S, 0, S.cnt[0], TILE, so0, ts),
                                     envelope_at(S, 1, S.cnt[1], TILE, so1, ts)), R(0.5));
            hnr = rsub(hr, mean);
        }
    } else {
#pragma unroll
        for (int r = 0; r < RW; ++r)
            hn[r] = v[r];
        hnl = hl;
        hnr = hr;
    }

    // Step 5 / Eq. (1): commit the IMF, update the residue, restart from it
    if (commit || mode == MODE_INIT) {
        R *imf = (R *)in.imf + (int64_t)imfc * in.imf_stride;
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int k = kbase + 32 * r;
            const bool inside = k < cnt;
            if (!(inside || (k == cnt && hasR)))
                continue;
            double rn = rsrc[k];
            if (commit) {
                const R c = hn[r];
                rn = __dsub_rn(rn, (double)c);
                if (inside) {
                    const int64_t p = ts + k;
                    int64_t dst;
                    if (in.imf_serialized)
                        imf[p] = c;
                    else if (deser_index(p, in.M, in.N, in.D, in.order, dst))
                        imf[dst] = c;
                    rdst[k] = rn;
                }
            }
            hn[r] = (R)rn;
        }
        if (tid == 0 && hasL)
            hnl = (R)(commit ? __dsub_rn(rsrc[-1], (double)hnl) : rsrc[-1]);
        if (tid == NT - 1 && hasR && cnt == TILE)
            hnr = (R)(commit ? __dsub_rn(rsrc[TILE], (double)hnr) : rsrc[TILE]);
    }

    // the new signal: edge values for the ENDPOINTS rule, SD partial sums
    if (!hasL && tid == 0)
        pa.taux[gt].h_first = (double)hn[0];
    if (!hasR) {
        const int kl = cnt - 1;
        if (kl >= kbase && ((kl - kbase) & 31) == 0 && (kl - kbase) / 32 < RW)
#pragma unroll
            for (int r = 0; r < RW; ++r)
                if (kbase + 32 * r == kl)
                    pa.taux[gt].h_last = (double)hn[r];
    }
    if (sift) {
        sdn = warp_sum(sdn);
        sdd = warp_sum(sdd);
        if (lane == 0) {
            S.red[0][warp] = sdn;
            S.red[1][warp] = sdd;
        }
    }

    // Step 1 on the new signal and the per-tile elimination of the spline system
    {
        uint32_t mx[RW], mn[RW];
        int wbase[2], pre[2][RW];
        detect_knots<R, TILE, NT>(S, hn, hnl, hnr, cnt, ts, L, mx, mn, wbase, pre);
        knot_slopes<R, TILE, NT>(S);
        __syncthreads();
    }
    if (warp < 2) {
        const int e = warp;
        const int m = S.cnt[e];
        TileExport *rec = pa.tex + 2 * (int64_t)gt + e;
        if (lane == 0) {
            rec->n = m;
            if (m >= 1) {
                const int ix[4] = {0, min(1, m - 1), max(m - 2, 0), m - 1};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    rec->t[q] = (int32_t)(ts + S.kt[e][sk(ix[q])]);
                    rec->y[q] = (double)S.ky[e][sk(ix[q])];
                }
            }
        }
        if (m >= 3) {
            const R xl[3] = {R(0), R(1), R(0)}, xr[3] = {R(0), R(0), R(1)};
            R f[3], l[3];
            warp_tridiag<R, 3, false>(
                m - 2, KnotRows<R>{S.kt[e], S.sl[e]}, xl, xr, S.cp[e], S.dp[e], S.bp[e],
                [](int, R) {}, f, l);
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    rec->xa[q] = (double)f[q];
                    rec->xb[q] = (double)l[q];
                }
            }
        }
    }
    if (sift && tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < NW; ++w) {
            a += S.red[0][w];
            b += S.red[1][w];
        }
        pa.taux[gt].sd_num = a;
        pa.taux[gt].sd_den = b;
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int k = kbase + 32 * r;
        if (k < cnt)
            hdst[k] = hn[r];
    }
    if (tid == 0 && pa.stats) {
        // algorithmic bytes per sample: h in (w) unless INIT, h out (w), and for a commit
        // the IMF out (w) and the residue in and out (16); INIT reads the residue (8)
        const unsigned long long w = sizeof(R);
        unsigned long long per = (mode == MODE_INIT) ? 8 + w : 2 * w;
        if (commit)
            per += w + 16;
        atomicAdd(&pa.stats->pass_bytes, per * (unsigned long long)cnt);
        if (sift)
            atomicAdd(&pa.stats->sample_sifts, (unsigned long long)cnt);
    }
}

// ---------------------------------------------------------------------------------
// Per instance: stop test and state machine, then the reduced interface system of
// the spline solve for each envelope (warp 0: maxima, warp 1: minima), in FP64.
__global__ void __launch_bounds__(64) k_reduce(ReduceArgs ra)
{
    const int ii = blockIdx.x;
    State *st = ra.state + ii;
    const int pm = st->mode;
    if (pm == MODE_DONE)
        return;
    const Inst &in = ra.inst[ii];
    const int e = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = in.ntiles, t0 = in.tile0;
    const int TQ = (nt + 31) / 32;
    const int ta = min(lane * TQ, nt), tb = min(ta + TQ, nt);
    int sn = 0, su = 0;
    for (int t = ta; t < tb; ++t) {
        const int n = ra.tex[2 * (int64_t)(t0 + t) + e].n;
        sn += n;
        su += min(n, 2);
    }
    int incl = su;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o)
            incl += y;
    }
    const int ubase = incl - su;
    const int U = __shfl_sync(FULLMASK, incl, 31);
    const int ntot = warp_sum(sn);
    __shared__ int s_ntot[2], s_next;
    __shared__ double s_sd[2];
    if (lane == 0)
        s_ntot[e] = ntot;
    if (e == 0) {
        double a = 0.0, b = 0.0;
        if (pm == MODE_SIFT)
            for (int t = ta; t < tb; ++t) {
                a += ra.taux[t0 + t].sd_num;
                b += ra.taux[t0 + t].sd_den;
            }
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) {
            s_sd[0] = a;
            s_sd[1] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nmax = s_ntot[0], nmin = s_ntot[1];
        const bool ok = nmax >= 1 && nmin >= 1 && nmax + nmin >= 3;
        State s = *st;
        s.hpar ^= 1;
        if (pm == MODE_SIFT_COMMIT || pm == MODE_COMMIT)
            s.rpar ^= 1;
        int nm;
        if (pm == MODE_INIT || pm == MODE_COMMIT || pm == MODE_SIFT_COMMIT) {
            if (pm != MODE_INIT) {
                s.sifts[s.imf_count] = s.sift_count + (pm == MODE_SIFT_COMMIT ? 1 : 0);
                s.imf_count += 1;
            }
            if (s.imf_count >= ra.K || !ok) {
                nm = MODE_DONE;
            } else {
                s.sift_count = 0;
                nm = (ra.stop == STOP_FIXED && ra.fixed_sifts == 1) ? MODE_SIFT_COMMIT : MODE_SIFT;
            }
        } else {
            s.sift_count += 1;
            if (!ok) {
                nm = MODE_COMMIT;
            } else if (ra.stop == STOP_FIXED) {
                nm = (s.sift_count >= ra.fixed_sifts - 1) ? MODE_SIFT_COMMIT : MODE_SIFT;
            } else {
                const double sd = s_sd[0] / s_sd[1];
                s.sd = sd;
                nm = (sd < ra.sd_threshold || s.sift_count >= ra.max_sifts) ? MODE_COMMIT
                                                                            : MODE_SIFT;
            }
        }
        s.nmax = nmax;
        s.nmin = nmin;
        s.mode = nm;
        *st = s;
        s_next = nm;
        if (nm != MODE_DONE)
            atomicAdd(ra.active, 1);
    }
    __syncthreads();
    const int nm = s_next;
    if (nm != MODE_SIFT && nm != MODE_SIFT_COMMIT)
        return;

    // reduced system: [left end knots][first/last knot of every non-empty tile][right end knots]
    REntry *Rn;
    double *A, *B, *C, *D, *Mv, *cpv, *dpv, *bpv;
    if (ra.smem_entries > 0) {
        // per envelope: cap REntry, then 8 double arrays of cap entries
        extern __shared__ __align__(16) unsigned char rsm[];
        const int64_t cap = ra.smem_entries;
        unsigned char *base = rsm + (size_t)e * (size_t)cap * (sizeof(REntry) + 8 * sizeof(double));
        Rn = reinterpret_cast<REntry *>(base);
        double *dbl = reinterpret_cast<double *>(base + (size_t)cap * sizeof(REntry));
        A = dbl;
        B = dbl + cap;
        C = dbl + 2 * cap;
        D = dbl + 3 * cap;
        Mv = dbl + 4 * cap;
        cpv = dbl + 5 * cap;
        dpv = dbl + 6 * cap;
        bpv = dbl + 7 * cap;
    } else {
        const int64_t rb = ra.rbase[ii] + (int64_t)e * skew_len(reduce_entries(nt));
        Rn = ra.rent + rb;
        A = ra.rA + rb;
        B = ra.rB + rb;
        C = ra.rC + rb;
        D = ra.rD + rb;
        Mv = ra.rM + rb;
        cpv = ra.rcp + rb;
        dpv = ra.rdp + rb;
        bpv = ra.rbp + rb;
    }
    const int nl = ra.boundary == BND_MIRROR ? min(ra.mirror_knots, ntot) : 1;
    const int nr = nl;
    const int NR = nl + U + nr;
    const TileExport *tex = ra.tex + 2 * (int64_t)t0 + e;
    {
        int p = nl + ubase;
        for (int t = ta; t < tb; ++t) {
            const TileExport &rc = tex[2 * (int64_t)t];
            if (rc.n == 1) {
                Rn[p++] = REntry{rc.t[0], t, RK_FL, 0, rc.y[0]};
            } else if (rc.n >= 2) {
                Rn[p++] = REntry{rc.t[0], t, RK_F, 0, rc.y[0]};
                Rn[p++] = REntry{rc.t[3], t, RK_L, 0, rc.y[3]};
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        const int64_t L = in.L;
        if (ra.boundary == BND_MIRROR) {
            // first two and last two knots of the whole signal, reflected about the ends
            const REntry k0 = Rn[nl];
            const TileExport &r0 = tex[2 * (int64_t)k0.tile];
            if (nl == 2) {
                int t1;
                double y1;
                if (r0.n >= 2) {
                    t1 = r0.t[1];
                    y1 = r0.y[1];
                } else {
                    t1 = Rn[nl + 1].t;
                    y1 = Rn[nl + 1].y;
                }
                Rn[0] = REntry{-t1, -1, RK_FIXED, 0, y1};
                Rn[1] = REntry{-k0.t, -1, RK_FREE, 0, k0.y};
            } else {
                Rn[0] = REntry{-k0.t, -1, RK_FIXED, 0, k0.y};
            }
            const REntry kl = Rn[nl + U - 1];
            const TileExport &rl = tex[2 * (int64_t)kl.tile];
            const int Lm = (int)(2 * (L - 1));
            if (nr == 2) {
                int t2;
                double y2;
                if (rl.n >= 2) {
                    t2 = rl.t[2];
                    y2 = rl.y[2];
                } else {
                    t2 = Rn[nl + U - 2].t;
                    y2 = Rn[nl + U - 2].y;
                }
                Rn[nl + U] = REntry{Lm - kl.t, -1, RK_FREE, 0, kl.y};
                Rn[nl + U + 1] = REntry{Lm - t2, -1, RK_FIXED, 0, y2};
            } else {
                Rn[nl + U] = REntry{Lm - kl.t, -1, RK_FIXED, 0, kl.y};
            }
        } else {
            Rn[0] = REntry{0, -1, RK_FIXED, 0, ra.taux[t0].h_first};
            Rn[nl + U] = REntry{(int)(L - 1), -1, RK_FIXED, 0, ra.taux[t0 + nt - 1].h_last};
        }
    }
    __syncwarp();
    // rows; a tile's interior knots next to its first/last knot are substituted by the
    // tile's elimination (M = x0 + u M_first + v M_last)
    for (int p = lane; p < NR; p += 32) {
        const REntry c = Rn[p];
        double a = 0.0, b = 1.0, cc = 0.0, d = 0.0;
        if (c.kind != RK_FIXED) {
            const REntry lf = Rn[p - 1], rg = Rn[p + 1];
            double tl = lf.t, yl = lf.y, tr = rg.t, yr = rg.y;
            const TileExport *rc = nullptr;
            if (c.kind == RK_F || c.kind == RK_L)
                rc = &tex[2 * (int64_t)c.tile];
            const bool subR = c.kind == RK_F && rc->n >= 3;
            const bool subL = c.kind == RK_L && rc->n >= 3;
            if (subR) {
                tr = rc->t[1];
                yr = rc->y[1];
            }
            if (subL) {
                tl = rc->t[2];
                yl = rc->y[2];
            }
            const double hl = (double)c.t - tl, hr = tr - (double)c.t;
            const double a0 = hl, b0 = 2.0 * (hl + hr), c0 = hr;
            const double d0 = 6.0 * ((yr - c.y) * rrcp(hr) - (c.y - yl) * rrcp(hl));
            a = a0;
            b = b0;
            cc = c0;
            d = d0;
            if (subR) {
                b = b0 + c0 * rc->xa[1];
                cc = c0 * rc->xa[2];
                d = d0 - c0 * rc->xa[0];
            }
            if (subL) {
                a = a0 * rc->xb[1];
                b = b0 + a0 * rc->xb[2];
                d = d0 - a0 * rc->xb[0];
            }
        }
        A[p] = a;
        B[p] = b;
        C[p] = cc;
        D[p] = d;
    }
    __syncwarp();
    {
        const double xl[1] = {0.0}, xr[1] = {0.0};
        double f1[1], l1[1];
        warp_tridiag<double, 1, true>(
            NR, ScratchRows{A, B, C, D}, xl, xr, cpv, dpv, bpv,
            [Mv](int i, double x) { Mv[i] = x; }, f1, l1);
    }
    __syncwarp();
    {
        int p = nl + ubase;
        for (int t = ta; t < tb; ++t) {
            const int n = tex[2 * (int64_t)t].n;
            const int u = min(n, 2);
            TileSolve so;
            const REntry pv = Rn[p - 1], nx = Rn[p + u];
            so.tp = pv.t;
            so.yp = pv.y;
            so.Mp = Mv[p - 1];
            so.tn = nx.t;
            so.yn = nx.y;
            so.Mn = Mv[p + u];
            so.MF = u >= 1 ? Mv[p] : 0.0;
            so.ML = u >= 1 ? Mv[p + u - 1] : 0.0;
            ra.tsol[2 * (int64_t)(t0 + t) + e] = so;
            p += u;
        }
    }
}

} // namespace semd
