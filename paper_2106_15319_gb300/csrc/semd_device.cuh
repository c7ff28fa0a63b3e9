// Device side of the GB300 Serial-EMD library: the sifting pass kernel, the interface
// solve of the partitioned spline system, and the warp-level tridiagonal machinery.
//
// Method (Zhang et al., arXiv 2106.15319): serialize the input (Sec. 3.2), sift the 1D
// signal (Sec. 2.1 Steps 1-5: extrema, cubic-spline envelopes, mean, subtract, stop
// test), commit IMFs (Eq. 1) and de-serialize (Sec. 3.3).
//
// Pass structure. Every instance's serialized signal is cut into tiles of TW = 32 * SPL
// samples; one warp owns one tile and each lane SPL consecutive samples. Warps never
// wait for one another: a CTA is only a group of independent warps. A pass reads the
// current signal h once and writes the next one once:
//   k_pass   (per tile)     - extrema of h as bit masks (Step 1), compaction of the knots
//                             into the warp's shared-memory pool, the tile's spline second
//                             derivatives given the tile-boundary values from the previous
//                             k_reduce (lanes 0-15 solve the maxima, lanes 16-31 the
//                             minima), envelope evaluation, mean and subtraction (Steps
//                             2-4), SD partial sums, IMF commit (Step 5 / Eq. 1); then the
//                             extrema of the new signal and the elimination of the tile's
//                             interior knots (the per-chunk part of the partitioned spline
//                             solve), exported as a short record.
//   k_reduce (per instance) - stop test and IMF state machine; then per envelope the
//                             reduced interface system (two unknowns per tile plus the end
//                             knots) in three levels: contiguous row segments eliminated in
//                             the working precision, the 32 segment-end unknowns solved in
//                             FP64 by cyclic reduction, the segments back-substituted;
//                             writes the tile-boundary values.
// Knot lists never leave shared memory: besides the signal, only ~100 bytes per tile
// and envelope cross HBM.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "semd_convert.cuh"
#include "semd_types.h"

namespace semd {

// Rounded arithmetic that the compiler may not contract into FMAs. Samples next to a
// tile edge are evaluated by two tiles (as a sample and as the neighbour's halo); both
// results must be bit-identical, so the envelope arithmetic uses explicit roundings.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
// Reciprocals: the hardware approximation in FP32 (the PTX rcp.approx instruction, about
// 1 ulp, denormal results flushed: every argument here is a knot spacing, a diagonal or a
// pivot of a diagonally dominant spline system, far from the denormal range); in FP64 that
// float seed refined by two Newton steps (about 1 ulp), which avoids the long IEEE division
// sequence on the narrow FP64 pipe. Both are deterministic, which is what the halo
// recomputation needs; neither is correctly rounded.
__device__ __forceinline__ float rrcp(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ double rrcp(double a)
{
    double r = (double)rrcp((float)a);
    double e = __fma_rn(-a, r, 1.0);
    r = __fma_rn(r, e, r);
    e = __fma_rn(-a, r, 1.0);
    return __fma_rn(r, e, r);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}

// Programmatic dependent launch: let the stream's next kernel start its CTAs now (they
// wait in pdl_wait), and wait until the previous kernel has completed and its writes are
// visible. Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Hint: fetch the line holding p into L1 (no register result).
__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// De-serialized destination of serialized sample p (Sec. 3.3): returns false for
// transition samples, which the de-serialization drops.
__device__ __forceinline__ bool deser_index(int64_t p, int64_t M, int64_t N, int64_t D, int order,
                                            int64_t &dst)
{
    // serialized lengths are below 2^30 (plan validation): 32-bit division
    const uint32_t md = (uint32_t)(M + D);
    const int64_t i = (uint32_t)p / md, m = p - i * (int64_t)md;
    if (m >= M)
        return false;
    dst = order == 0 ? i * M + m : m * N + i;
    return true;
}

// ---------------------------------------------------------------------------------
// Partitioned tridiagonal solve.
//
// Unknowns x_0..x_{n-1}; row i: a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i, with the
// outside values x_{-1} = xl[col] and x_n = xr[col] given per right-hand-side column.
// Column 0 carries d; columns 1.. have d = 0 (they give the response to the outside
// values). Worker l owns rows [s, e); it eliminates rows s..e-2 with the Thomas
// algorithm in terms of x_{s-1} (last unknown of worker l-1) and x_{e-1} (its own last
// unknown Z_l), which leaves one reduced row per worker coupling Z_{l-1}, Z_l, Z_{l+1}.
// The matrix is diagonally dominant (spline rows: b = 2(a + c)), so no pivoting is
// needed.

// Per-worker result of the segment elimination: x_s = alS + beS x_{s-1} + gaS Z_l,
// x_{e-2} = alE + beE x_{s-1} + gaE Z_l, and the worker's last row (al, bl, cl, dl).
template <typename R>
struct SegElim {
    R alS = R(0), beS = R(0), gaS = R(1), alE = R(0), beE = R(1), gaE = R(0);
    R al = R(0), bl = R(1), cl = R(0), dl = R(0);
};

// Parallel cyclic reduction of one tridiagonal row per lane over groups of W lanes
// (A Z_{l-1} + B Z_l + C Z_{l+1} = D[k]; A = 0 on a group's first lane, C = 0 on its
// last): log2(W) steps of shuffles; returns Z per right-hand-side column. At step st the
// coupling of a lane to a partner st lanes outside its group is already exactly zero (A
// for the first st lanes, C for the last st), and a shuffle from outside the group
// returns the lane's own, finite values, so no masking is needed.
template <typename R, int NCOL, int W>
__device__ __forceinline__ void pcr_solve(R A, R B, R C, R (&D)[NCOL], R (&Z)[NCOL])
{
#pragma unroll
    for (int st = 1; st < W; st <<= 1) {
        // the neighbours' diagonals enter only through their reciprocals: one per lane
        const R iB = rrcp(B);
        const R Am = __shfl_up_sync(FULLMASK, A, st, W), iBm = __shfl_up_sync(FULLMASK, iB, st, W);
        const R Cm = __shfl_up_sync(FULLMASK, C, st, W);
        const R Ap = __shfl_down_sync(FULLMASK, A, st, W), iBp = __shfl_down_sync(FULLMASK, iB, st, W);
        const R Cp = __shfl_down_sync(FULLMASK, C, st, W);
        R Dm[NCOL], Dp[NCOL];
#pragma unroll
        for (int k = 0; k < NCOL; ++k) {
            Dm[k] = __shfl_up_sync(FULLMASK, D[k], st, W);
            Dp[k] = __shfl_down_sync(FULLMASK, D[k], st, W);
        }
        const R k1 = A * iBm, k2 = C * iBp;
        const R nA = -k1 * Am, nC = -k2 * Cp, nB = B - k1 * Cm - k2 * Ap;
#pragma unroll
        for (int k = 0; k < NCOL; ++k)
            D[k] = D[k] - k1 * Dm[k] - k2 * Dp[k];
        A = nA;
        B = nB;
        C = nC;
    }
    const R invB = rrcp(B);
#pragma unroll
    for (int k = 0; k < NCOL; ++k)
        Z[k] = D[k] * invB;
}

// One column of pcr_solve that also keeps its elimination factors, so that a further
// right-hand side of the same rows is solved by pcr_apply with the shuffles of D alone:
// pcr_apply performs the same operations on D as pcr_solve, with the same result.
template <typename R, int W>
struct PcrFactors {
    static constexpr int kSteps = W >= 32 ? 5 : W >= 16 ? 4 : W >= 8 ? 3 : W >= 4 ? 2 : 1;
    R k1[kSteps], k2[kSteps], invB;
};
template <typename R, int W>
__device__ __forceinline__ R pcr_solve_keep(R A, R B, R C, R D, PcrFactors<R, W> &f)
{
    int i = 0;
#pragma unroll
    for (int st = 1; st < W; st <<= 1, ++i) {
        const R iB = rrcp(B);
        const R Am = __shfl_up_sync(FULLMASK, A, st, W), iBm = __shfl_up_sync(FULLMASK, iB, st, W);
        const R Cm = __shfl_up_sync(FULLMASK, C, st, W);
        const R Ap = __shfl_down_sync(FULLMASK, A, st, W), iBp = __shfl_down_sync(FULLMASK, iB, st, W);
        const R Cp = __shfl_down_sync(FULLMASK, C, st, W);
        const R Dm = __shfl_up_sync(FULLMASK, D, st, W), Dp = __shfl_down_sync(FULLMASK, D, st, W);
        const R k1 = A * iBm, k2 = C * iBp;
        const R nA = -k1 * Am, nC = -k2 * Cp, nB = B - k1 * Cm - k2 * Ap;
        D = D - k1 * Dm - k2 * Dp;
        A = nA;
        B = nB;
        C = nC;
        f.k1[i] = k1;
        f.k2[i] = k2;
    }
    f.invB = rrcp(B);
    return D * f.invB;
}
template <typename R, int W>
__device__ __forceinline__ R pcr_apply(const PcrFactors<R, W> &f, R D)
{
    int i = 0;
#pragma unroll
    for (int st = 1; st < W; st <<= 1, ++i) {
        const R Dm = __shfl_up_sync(FULLMASK, D, st, W), Dp = __shfl_down_sync(FULLMASK, D, st, W);
        D = D - f.k1[i] * Dm - f.k2[i] * Dp;
    }
    return D * f.invB;
}

// Reduced row of a worker from its segment elimination g and the next worker's
// first-unknown expression (nalS, nbeS, ngaS): A Z_{l-1} + B Z_l + C Z_{l+1} = D.
// Workers without rows (q == 0) get the dummy row Z = 0.
template <typename R>
__device__ __forceinline__ void reduced_row(const SegElim<R> &g, int q, bool has_next, R nalS,
                                            R nbeS, R ngaS, R &A, R &B, R &C, R &D)
{
    A = R(0);
    B = R(1);
    C = R(0);
    D = R(0);
    if (q >= 1) {
        A = g.al * g.beE;
        B = g.bl + g.al * g.gaE + (has_next ? g.cl * nbeS : R(0));
        C = has_next ? g.cl * ngaS : R(0);
        D = g.dl - g.al * g.alE - (has_next ? g.cl * nalS : R(0));
    }
}

// The reduced system of W lanes (W = 16: the two half-warps solve two independent
// systems in the same instructions; W = 2, 4, 8 for small systems) with the outside
// values xl (before the first lane's rows) and xr (after the last rows), solved by
// cyclic reduction; returns Z_l per column (dummy 0 for lanes without rows).
template <typename R, int NCOL, int W>
__device__ __forceinline__ void warp_reduced_solve(const SegElim<R> &g, int q, bool has_next,
                                                   const R (&xl)[NCOL], const R (&xr)[NCOL],
                                                   R (&Z)[NCOL])
{
    const int wl = threadIdx.x & (W - 1);
    const R nalS = __shfl_down_sync(FULLMASK, g.alS, 1, W);
    const R nbeS = __shfl_down_sync(FULLMASK, g.beS, 1, W);
    const R ngaS = __shfl_down_sync(FULLMASK, g.gaS, 1, W);
    R A, B, C, D[NCOL];
    reduced_row(g, q, has_next, nalS, nbeS, ngaS, A, B, C, D[0]);
#pragma unroll
    for (int k = 1; k < NCOL; ++k)
        D[k] = R(0);
    if (q >= 1) {
        if (wl == 0) {
#pragma unroll
            for (int k = 0; k < NCOL; ++k)
                D[k] -= A * xl[k];
            A = R(0);
        }
        if (!has_next) {
#pragma unroll
            for (int k = 0; k < NCOL; ++k)
                D[k] -= g.cl * xr[k];
        }
    }
    pcr_solve<R, NCOL, W>(A, B, C, D, Z);
}

// ---------------------------------------------------------------------------------
// Envelope cubics. Interval (tl, tr) with values (yl, yr) and second derivatives
// (Ml, Mr) is stored as the local polynomial e(u) = c0 + c1 u + c2 u^2 + c3 u^3,
// u = k - tl: the textbook interval formula of the natural cubic spline expanded in
// powers of u. Coefficients are pre-multiplied by 1/2 (exact in binary floating point),
// so the mean envelope of Step 3 is the plain sum of the two evaluations.
template <typename R>
struct __align__(16) Coef {
    R c0, c1, c2, c3;
};

template <typename R>
__device__ __forceinline__ Coef<R> half_cubic_from(R yl, R Ml, R Mr, R h, R inv, R slope)
{
    Coef<R> c;
    c.c0 = rmul(yl, R(0.5));
    c.c1 = rmul(rsub(slope, rmul(rmul(h, radd(rmul(R(2), Ml), Mr)), R(1.0 / 6.0))), R(0.5));
    c.c2 = rmul(Ml, R(0.25));
    c.c3 = rmul(rmul(rsub(Mr, Ml), inv), R(1.0 / 12.0));
    return c;
}

template <typename R>
__device__ __forceinline__ Coef<R> half_cubic(int tl, R yl, R Ml, int tr, R yr, R Mr)
{
    const R h = R(tr - tl);
    const R inv = rrcp(h);
    return half_cubic_from(yl, Ml, Mr, h, inv, rmul(rsub(yr, yl), inv));
}

template <typename R>
__device__ __forceinline__ R horner(const Coef<R> &c, R u)
{
    return rfma(rfma(rfma(c.c3, u, c.c2), u, c.c1), u, c.c0);
}

// ---------------------------------------------------------------------------------
// Shared memory of one warp tile: a pool of knot slots shared by both envelopes.
// Maxima use slots [0, m0 + 2), minima [m0 + 2, m0 + m1 + 4). Within an envelope's range,
// slot 0 is the bracket knot before the tile, slot j + 1 knot j, slot m + 1 the bracket
// knot after it; ky holds each slot's position (tile-relative) and value, cf[q] the
// interval whose left knot sits in slot q (interval q = knot q-1 -> knot q), rw the
// elimination of row i (knot i + 1) at slot i. Every sample is at most one kind of
// extremum, so m0 + m1 <= TW.
template <typename R>
struct __align__(8) KnotY {
    int t;
    R y;
};
template <>
struct __align__(16) KnotY<double> {
    int t;
    double y;
};
template <typename R, int TW>
struct WarpPool {
    static constexpr int KP = TW + 4;
    Coef<R> cf[KP];
    Coef<R> rw[KP];
    KnotY<R> ky[KP];
};

// A warp's next tile, copied in while the current one computes (staging kernels only,
// placed after the warps' pools): the signal (zero past the tile's count), the halo
// samples before and after it, and both envelopes' interface values.
template <typename R, int TW>
struct StageBuf {
    R stage[TW + 16 / sizeof(R)];
    TileSolve sts[2];
    uint2 km[32]; // the signal's extremum masks and ranks, per lane
};

// The interface solution of one tile and envelope in the working precision (FP32 pass
// kernels read the single-precision values, so they issue no FP64 conversions).
template <typename R>
struct SolveVals {
    R MF, ML, yp, Mp, yn, Mn, M1, M2;
};
__device__ __forceinline__ SolveVals<float> solve_vals(const TileSolve &so, float)
{
    const float4 a = *reinterpret_cast<const float4 *>(&so.f[0]);
    const float4 b = *reinterpret_cast<const float4 *>(&so.f[4]);
    return {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}
__device__ __forceinline__ SolveVals<double> solve_vals(const TileSolve &so, double)
{
    return {so.MF, so.ML, so.yp, so.Mp, so.yn, so.Mn, so.M1, so.M2};
}

// Second derivative of knot j of an envelope with m <= kSparseKnots knots, all of which
// the interface solve determined.
template <typename R>
__device__ __forceinline__ R sparse_M(const SolveVals<R> &sv, int j, int m)
{
    return j == 0 ? sv.MF : (j == m - 1 ? sv.ML : (j == 1 ? sv.M1 : sv.M2));
}

// N consecutive values through 16-byte vector accesses (p 16-byte aligned).
template <int N>
__device__ __forceinline__ void vload(const float *p, float (&v)[N])
{
    static_assert(N % 4 == 0, "whole float4s");
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        const float4 a = reinterpret_cast<const float4 *>(p)[i];
        v[4 * i] = a.x;
        v[4 * i + 1] = a.y;
        v[4 * i + 2] = a.z;
        v[4 * i + 3] = a.w;
    }
}
template <int N>
__device__ __forceinline__ void vload(const double *p, double (&v)[N])
{
    static_assert(N % 2 == 0, "whole double2s");
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const double2 a = reinterpret_cast<const double2 *>(p)[i];
        v[2 * i] = a.x;
        v[2 * i + 1] = a.y;
    }
}
template <int N>
__device__ __forceinline__ void vstore(float *p, const float (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
        reinterpret_cast<float4 *>(p)[i] =
            make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
template <int N>
__device__ __forceinline__ void vstore(double *p, const double (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N / 2; ++i)
        reinterpret_cast<double2 *>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// N consecutive samples starting at k0, zero at and past cnt. p + k0 is 16-byte aligned.
template <typename T, int N>
__device__ __forceinline__ void loadn(const T *p, int k0, int cnt, T (&v)[N])
{
    if (k0 + N <= cnt) {
        vload<N>(p + k0, v);
    } else {
#pragma unroll
        for (int s = 0; s < N; ++s)
            v[s] = (k0 + s < cnt) ? p[k0 + s] : T(0);
    }
}

template <typename T, int N>
__device__ __forceinline__ void storen(T *p, int k0, int cnt, const T (&v)[N])
{
    if (k0 + N <= cnt) {
        vstore<N>(p + k0, v);
    } else {
#pragma unroll
        for (int s = 0; s < N; ++s)
            if (k0 + s < cnt)
                p[k0 + s] = v[s];
    }
}

// The same loads cached in L2 only (not L1): for data another kernel wrote while this one
// was already resident.
template <int N>
__device__ __forceinline__ void vload_cg(const float *p, float (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        const float4 a = __ldcg(reinterpret_cast<const float4 *>(p) + i);
        v[4 * i] = a.x;
        v[4 * i + 1] = a.y;
        v[4 * i + 2] = a.z;
        v[4 * i + 3] = a.w;
    }
}
template <int N>
__device__ __forceinline__ void vload_cg(const double *p, double (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const double2 a = __ldcg(reinterpret_cast<const double2 *>(p) + i);
        v[2 * i] = a.x;
        v[2 * i + 1] = a.y;
    }
}
template <typename T, int N>
__device__ __forceinline__ void loadn_cg(const T *p, int k0, int cnt, T (&v)[N])
{
    if (k0 + N <= cnt) {
        vload_cg<N>(p + k0, v);
    } else {
#pragma unroll
        for (int s = 0; s < N; ++s)
            v[s] = (k0 + s < cnt) ? __ldcg(p + k0 + s) : T(0);
    }
}

// Knots (tile position and value) of this lane's samples into the pool in rank order:
// maxima at slots 1 + bx.., minima at slots m0 + 3 + bn...
// A sample is at most one kind of extremum, so each sample takes at most one store: the
// slot of its kind's next knot.
template <typename R, int SPL, int TW>
__device__ __forceinline__ void knot_compact(WarpPool<R, TW> &P, const R (&v)[SPL], int k0,
                                             uint32_t MX, uint32_t MN, int bx, int bn, int m0)
{
    int ix = 1 + bx, in = m0 + 3 + bn;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
        const int px = (int)((MX >> s) & 1u), pn = (int)((MN >> s) & 1u);
        if (px | pn)
            P.ky[px ? ix : in] = KnotY<R>{k0 + s, v[s]};
        ix += px;
        in += pn;
    }
}

// Step 1 on one warp tile: extremum masks of this lane's SPL samples (maximum:
// h[k-1] < h[k] >= h[k+1]; minimum: h[k-1] > h[k] <= h[k+1]; never at the instance's
// end samples), their warp-wide exclusive ranks (bx, bn), the counts (m0, m1), and the
// knots (tile position and value) compacted into the pool: maxima at slots 1.., minima
// at slots m0 + 3... `left` / `right` are the samples next to this lane's run.
template <typename R, int SPL, int TW>
__device__ __forceinline__ void warp_knots(WarpPool<R, TW> &P, const R (&v)[SPL], R left, R right,
                                           int k0, int g0, int cnt, int L, uint32_t &MX,
                                           uint32_t &MN, int &bx, int &bn, int &m0, int &m1)
{
    const int lane = threadIdx.x & 31;
    uint32_t up = 0, dn = 0; // bit s: h[k0+s] < h[k0+s+1] / h[k0+s] > h[k0+s+1]
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
        const R nx = s < SPL - 1 ? v[s + 1] : right;
        up |= (uint32_t)(v[s] < nx) << s;
        dn |= (uint32_t)(v[s] > nx) << s;
    }
    const uint32_t upl = (up << 1) | (uint32_t)(left < v[0]);
    const uint32_t dnl = (dn << 1) | (uint32_t)(left > v[0]);
    // valid samples: inside the tile's count and 1 <= instance index <= L-2
    const int lo = max(0, 1 - g0), hi = min(min(SPL, cnt - k0), L - 1 - g0);
    const uint32_t valid = hi > lo ? (((2u << (hi - 1)) - 1u) & ~((1u << lo) - 1u)) : 0u;
    MX = upl & ~up & valid;
    MN = dnl & ~dn & valid;
    const uint32_t packed = (uint32_t)__popc(MX) | ((uint32_t)__popc(MN) << 16);
    uint32_t incl = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o)
            incl += y;
    }
    const uint32_t total = __shfl_sync(FULLMASK, incl, 31);
    const uint32_t before = incl - packed;
    bx = (int)(before & 0xffffu);
    bn = (int)(before >> 16);
    m0 = (int)(total & 0xffffu);
    m1 = (int)(total >> 16);
    knot_compact<R, SPL, TW>(P, v, k0, MX, MN, bx, bn, m0);
}

// The same from masks and ranks a previous pass stored for this signal (packed per lane:
// x = MX | MN << 16, y = bx | bn << 16), without the comparisons and the scan.
template <typename R, int SPL, int TW>
__device__ __forceinline__ void warp_knots_stored(WarpPool<R, TW> &P, const R (&v)[SPL], int k0,
                                                  uint2 km, uint32_t &MX, uint32_t &MN, int &bx,
                                                  int &bn, int &m0, int &m1)
{
    MX = km.x & 0xffffu;
    MN = km.x >> 16;
    bx = (int)(km.y & 0xffffu);
    bn = (int)(km.y >> 16);
    m0 = __shfl_sync(FULLMASK, bx + __popc(MX), 31);
    m1 = __shfl_sync(FULLMASK, bn + __popc(MN), 31);
    knot_compact<R, SPL, TW>(P, v, k0, MX, MN, bx, bn, m0);
}

// Forward elimination of the interior spline rows s..e-1 of one envelope (row i: knot
// i + 1, pool slot i + 2; h_q, S_q length and slope of interval q):
//   h_{i+1} M_i + 2 (h_{i+1} + h_{i+2}) M_{i+1} + h_{i+2} M_{i+2} = 6 (S_{i+2} - S_{i+1}),
// rows s..e-2 in terms of x_{s-1} and the segment's last unknown x_{e-1} (kept as the
// lane's last row), then the backward sweep to the segment's first unknown.
// With STORE_IV, also stores every interval's (slope, 1/length, length, left value) in
// IV[q], for the cubics of the back-substitution.
template <typename R, bool STORE_IV>
__device__ __forceinline__ void seg_forward(const KnotY<R> *K, Coef<R> *RW, Coef<R> *IV, int s,
                                            int e, SegElim<R> &g)
{
    if (e <= s)
        return;
    // length and slope of interval s + 1 (slots s + 1 -> s + 2)
    const KnotY<R> k0 = K[s + 1];
    KnotY<R> kB = K[s + 2];
    R hA = R(kB.t - k0.t);
    R iA = rrcp(hA);
    R SA = (kB.y - k0.y) * iA;
    if (STORE_IV)
        IV[s + 1] = Coef<R>{SA, iA, hA, k0.y};
    // carried terms of the previous row; their start values make the first row's
    // elimination plain (den = b, dp = d / b, bp = -a / b)
    R cprev = R(0), dprev = R(0), bprev = R(1);
    for (int j = s; j < e; ++j) {
        const KnotY<R> kN = K[j + 3];
        const R hB = R(kN.t - kB.t);
        const R iB = rrcp(hB);
        const R SB = (kN.y - kB.y) * iB;
        if (STORE_IV)
            IV[j + 2] = Coef<R>{SB, iB, hB, kB.y};
        const R a = hA, c = hB, b = R(2) * (a + c), d = R(6) * (SB - SA);
        if (j < e - 1) {
            const R inv = rrcp(b - a * cprev);
            cprev = c * inv;
            dprev = (d - a * dprev) * inv;
            bprev = -a * bprev * inv;
            RW[j] = Coef<R>{cprev, dprev, bprev, R(0)};
        } else {
            g.al = a;
            g.bl = b;
            g.cl = c;
            g.dl = d;
        }
        kB = kN;
        hA = hB;
        SA = SB;
    }
    if (e - s >= 2) {
        g.alE = dprev;
        g.beE = bprev;
        g.gaE = -cprev;
        R xa = g.alE, xb = g.beE, xg = g.gaE;
        for (int r = e - 3; r >= s; --r) {
            const Coef<R> w = RW[r];
            xa = w.c1 - w.c0 * xa;
            xb = w.c2 - w.c0 * xb;
            xg = -w.c0 * xg;
        }
        g.alS = xa;
        g.beS = xb;
        g.gaS = xg;
    }
}

// Halved cubic of the interval whose left knot is slot q.
template <typename R>
__device__ __forceinline__ Coef<R> slot_cubic(const KnotY<R> *K, int q, R Ml, R Mr)
{
    const KnotY<R> a = K[q], b = K[q + 1];
    return half_cubic<R>(a.t, a.y, Ml, b.t, b.y, Mr);
}


// Step 2 for one envelope of the tile (one half-warp, lane hl of 16), then the halved
// cubic of every interval q = 0..m into cf. An envelope with at most kSparseKnots knots
// has every knot's second derivative from the interface solve (lane hl writes interval
// hl). A denser one solves for its interior knots 1..m-2 given M_0 = MF and M_{m-1} = ML:
// each lane eliminates a run of Q rows, cyclic reduction over W-lane groups joins the
// runs, back-substitution writes the cubics. The end intervals (to the bracket knots)
// use half_cubic on values both neighbouring tiles hold bit for bit, so a sample next to
// a tile edge evaluates identically in both. Called by all 32 lanes (the shuffles span
// the warp); run_pcr (warp-uniform) tells whether either envelope is dense.
template <typename R, int TW, int W>
__device__ __forceinline__ void env_solve(WarpPool<R, TW> &P, int base, int m, int hl, int Q,
                                          const SolveVals<R> &sv, bool run_pcr)
{
    const KnotY<R> *K = P.ky + base;
    Coef<R> *CF = P.cf + base;
    Coef<R> *RW = P.rw + base;
    const R MF = sv.MF, ML = sv.ML;
    const bool sparse = m <= kSparseKnots;
    if (sparse) {
        if (hl <= m) {
            const R Ml = hl == 0 ? sv.Mp : sparse_M(sv, hl - 1, m);
            const R Mr = hl == m ? sv.Mn : sparse_M(sv, hl, m);
            CF[hl] = slot_cubic(K, hl, Ml, Mr);
        }
    } else if (hl == 0) {
        CF[0] = slot_cubic(K, 0, sv.Mp, MF);
        CF[m] = slot_cubic(K, m, ML, sv.Mn);
    }
    if (!run_pcr)
        return;
    const int n = sparse ? 0 : m - 2; // interior unknowns; row i is knot i + 1 (slot i + 2)
    const int s = min(hl * Q, n), e = min(s + Q, n), q = e - s;
    SegElim<R> g;
    seg_forward<R, true>(K, RW, CF, s, e, g);
    __syncwarp(); // a neighbour's forward sweep wrote interval data this lane reads below
    const R xl[1] = {MF}, xr[1] = {ML};
    R Z[1];
    warp_reduced_solve<R, 1, W>(g, q, (q >= 1) && (e < n), xl, xr, Z);
    R Zp = __shfl_up_sync(FULLMASK, Z[0], 1, W);
    if (hl == 0)
        Zp = MF;
    if (q >= 1) {
        // back-substitution, descending; the interval with left slot j + 2 (knot j + 1 ->
        // j + 2) is written as soon as both of its second derivatives are known
        auto cubic = [&](int qq, R Ml, R Mr) {
            const Coef<R> iv = CF[qq];
            CF[qq] = half_cubic_from(iv.c3, Ml, Mr, iv.c2, iv.c1, iv.c0);
        };
        R xn = Z[0];
        if (e == n)
            cubic(n + 1, xn, ML);
        for (int j = e - 2; j >= s; --j) {
            const Coef<R> w = RW[j];
            const R x = w.c1 + w.c2 * Zp - w.c0 * xn;
            cubic(j + 2, x, xn);
            xn = x;
        }
        cubic(s + 1, Zp, xn);
    }
}

// Elimination of the interior of a dense envelope of the tile (one half-warp) in terms
// of the unknown M_0 and M_{m-1}: M_1 = first[0] + first[1] M_0 + first[2] M_{m-1} and
// M_{m-2} likewise (last). A sparse envelope takes part as empty rows. Called by all 32
// lanes (or by none).
template <typename R, int TW, int W>
__device__ __forceinline__ void env_export(WarpPool<R, TW> &P, int base, int m, int hl, int Q,
                                           R (&first)[3], R (&last)[3])
{
    const int n = m <= kSparseKnots ? 0 : m - 2;
    const int s = min(hl * Q, n), e = min(s + Q, n), q = e - s;
    SegElim<R> g;
    seg_forward<R, false>(P.ky + base, P.rw + base, nullptr, s, e, g);
    const R xl[3] = {R(0), R(1), R(0)}, xr[3] = {R(0), R(0), R(1)};
    R Z[3];
    warp_reduced_solve<R, 3, W>(g, q, (q >= 1) && (e < n), xl, xr, Z);
    const int last_lane = n > 0 ? (n - 1) / Q : 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const R f = (k == 0 ? g.alS : R(0)) + g.beS * xl[k] + g.gaS * Z[k];
        first[k] = __shfl_sync(FULLMASK, f, 0, W);
        last[k] = __shfl_sync(FULLMASK, Z[k], last_lane, W);
    }
}

// Interior unknowns of the denser of the tile's two envelopes (0 when both are sparse).
__device__ __forceinline__ int dense_rows(int m0, int m1)
{
    const int d0 = m0 > kSparseKnots ? m0 - 2 : 0, d1 = m1 > kSparseKnots ? m1 - 2 : 0;
    return max(d0, d1);
}

// The solves with the narrowest lane group that covers the denser envelope's interior
// with one row per lane (W = 4, 8), else all 16 lanes of the half-warp (Q rows per lane,
// Q odd so the lanes hit distinct banks): cyclic reduction takes log2(W) steps.
template <typename R, int TW>
__device__ __forceinline__ void env_solve_any(WarpPool<R, TW> &P, int base, int m, int hl, int m0,
                                              int m1, const SolveVals<R> &sv)
{
    const int nmax = dense_rows(m0, m1);
    if (nmax == 0)
        env_solve<R, TW, 4>(P, base, m, hl, 1, sv, false);
    else if (nmax <= 4)
        env_solve<R, TW, 4>(P, base, m, hl, 1, sv, true);
    else if (nmax <= 8)
        env_solve<R, TW, 8>(P, base, m, hl, 1, sv, true);
    else
        env_solve<R, TW, 16>(P, base, m, hl, ((nmax + 15) >> 4) | 1, sv, true);
}

template <typename R, int TW>
__device__ __forceinline__ void env_export_any(WarpPool<R, TW> &P, int base, int m, int hl, int m0,
                                               int m1, R (&first)[3], R (&last)[3])
{
    const int nmax = dense_rows(m0, m1);
    if (nmax <= 4)
        env_export<R, TW, 4>(P, base, m, hl, 1, first, last);
    else if (nmax <= 8)
        env_export<R, TW, 8>(P, base, m, hl, 1, first, last);
    else
        env_export<R, TW, 16>(P, base, m, hl, ((nmax + 15) >> 4) | 1, first, last);
}

// Whole-record 16-byte accesses to the tile records.
template <typename R>
union RecWords {
    int4 v[sizeof(TileRec<R>) / 16];
    TileRec<R> r;
};
template <typename R>
__device__ __forceinline__ void store_rec(TileRec<R> *p, const TileRec<R> &r)
{
    RecWords<R> u;
    u.r = r;
#pragma unroll
    for (int i = 0; i < (int)(sizeof(TileRec<R>) / 16); ++i)
        reinterpret_cast<int4 *>(p)[i] = u.v[i];
}
template <typename R>
__device__ __forceinline__ TileRec<R> load_rec(const TileRec<R> *p)
{
    RecWords<R> u;
#pragma unroll
    for (int i = 0; i < (int)(sizeof(TileRec<R>) / 16); ++i)
        u.v[i] = reinterpret_cast<const int4 *>(p)[i];
    return u.r;
}

// Asynchronous global -> shared copies (no registers held while in flight): 16 bytes of
// which the first src_bytes are read and the rest zero-filled (both addresses 16-byte
// aligned; src is read only when src_bytes > 0), or one 4- or 8-byte element.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_elem(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double *dst, const double *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Asks L2 to fetch [p, p + bytes) ahead of use (p 16-byte aligned, bytes a multiple of
// 16, the range inside one allocation). No completion is awaited.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Starts the copy of tile gt's inputs into the warp's stage buffer (all 32 lanes): the
// signal (SPL samples per lane, 16-byte chunks, zero past the tile's count), the halo
// samples next to it, and for a sifting mode both envelopes' interface values. Tiles
// whose mode reads no signal (INIT, DONE) are not staged. Returns whether it copied.
template <typename R, int SPL>
__device__ __forceinline__ void stage_issue(StageBuf<R, 32 * SPL> &P, int mode, const R *hsrc,
                                            int ts, int L, const TileSolve *tsol,
                                            const uint2 *kmask, int ntiles, int lt)
{
    constexpr int TW = 32 * SPL;
    constexpr int PER = 16 / (int)sizeof(R); // samples per 16-byte chunk
    const int lane = threadIdx.x & 31;
    const int cnt = min(TW, L - ts);
    const int k0 = lane * SPL;
#pragma unroll
    for (int c = 0; c < SPL / PER; ++c) {
        const int k = k0 + c * PER;
        const int valid = max(0, min(PER, cnt - k));
        cp_async16(&P.stage[k], valid > 0 ? hsrc + k : hsrc, valid * (int)sizeof(R));
    }
    if (lane == 0 && ts > 0)
        cp_async_elem(&P.stage[TW], hsrc - 1);
    if (lane == 31 && ts + TW < L)
        cp_async_elem(&P.stage[TW + 1], hsrc + TW);
    if (mode == MODE_SIFT || mode == MODE_SIFT_COMMIT) {
        if (lane < 14) {
            constexpr int CH = (int)sizeof(TileSolve) / 16; // 7 chunks per envelope
            const int e = lane / CH, q = lane - e * CH;
            const char *src = reinterpret_cast<const char *>(tsol + (int64_t)e * ntiles + lt);
            cp_async16(reinterpret_cast<char *>(&P.sts[e]) + 16 * q, src + 16 * q, 16);
        }
        cp_async8(&P.km[lane], kmask + (int64_t)lt * 32 + lane);
    }
    cp_async_commit();
}

// The same for a tile of another instance than the current one (its descriptor and state
// read first).
template <typename R, int SPL>
__device__ __forceinline__ bool stage_tile(const PassArgs &pa, StageBuf<R, 32 * SPL> &P,
                                           int64_t gt)
{
    constexpr int TW = 32 * SPL;
    const int ii = pa.tile_inst[gt];
    const State *stp = pa.state + ii;
    const int mode = stp->mode;
    if (mode == MODE_DONE || mode == MODE_INIT)
        return false;
    const Inst &in = pa.inst[ii];
    const int lt = (int)(gt - in.tile0);
    const int ts = lt * TW;
    stage_issue<R, SPL>(P, mode, (const R *)in.h[stp->hpar] + ts, ts, (int)in.L, in.tsol,
                        in.kmask, in.ntiles, lt);
    return true;
}

// A warp's first tile, read before the pass kernel waits for the interface solve: the
// signal, its halo samples and its stored extremum masks, which the previous pass wrote.
// The interface solve, the kernel before this one, lets it start only once it has itself
// waited for that pass (so those writes are complete); the loads bypass L1. The signal
// buffer is predicted from the previous pass's parity (the interface solve flips it after
// every pass); the pass uses these values only if the prediction holds and the tile sifts
// or commits.
template <typename R, int SPL>
struct PreTile {
    R v[SPL];
    R hcl, hcr;
    uint2 km;
    int hpar;
    // the knots compacted into the warp's pool from km (warp_knots_stored), and its results;
    // ok: the compaction ran (every slot the masks imply lies inside the pool)
    uint32_t MX, MN;
    int bx, bn, m0, m1;
    bool ok;
};
template <typename R, int SPL>
__device__ __forceinline__ void pre_tile(const PassArgs &pa, int64_t gt, PreTile<R, SPL> &pt,
                                         WarpPool<R, 32 * SPL> &P)
{
    constexpr int TW = 32 * SPL;
    const int lane = threadIdx.x & 31;
    const int ii = pa.tile_inst[gt];
    const Inst &in = pa.inst[ii];
    const int ppar = __shfl_sync(FULLMASK, __ldcg(&pa.state[ii].pass_par), 0);
    pt.hpar = (ppar & 1) ^ 1;
    const int L = (int)in.L, lt = (int)(gt - in.tile0), ts = lt * TW;
    const int cnt = min(TW, L - ts);
    const R *hsrc = (const R *)in.h[pt.hpar] + ts;
    loadn_cg<R, SPL>(hsrc, lane * SPL, cnt, pt.v);
    pt.hcl = (lane == 0 && ts > 0) ? __ldcg(hsrc - 1) : R(0);
    pt.hcr = (lane == 31 && ts + TW < L) ? __ldcg(hsrc + TW) : R(0);
    pt.km = __ldcg(in.kmask + (int64_t)lt * 32 + lane);
    // Step 1's knots of this signal into the pool now (used if the tile sifts). Before the
    // wait the stored masks may belong to another signal (an instance that starts with
    // this pass, an earlier call with another tile size) or may never have been written,
    // so the knots are compacted only if every slot the masks and ranks imply lies inside
    // the pool, which masks of this signal always satisfy (bx + |MX| <= m0 and
    // m0 + bn + |MN| <= m0 + m1 <= TW); otherwise the pass compacts after its wait.
    const uint32_t MX = pt.km.x & 0xffffu, MN = pt.km.x >> 16;
    const int bx = (int)(pt.km.y & 0xffffu), bn = (int)(pt.km.y >> 16);
    const int m0 = __shfl_sync(FULLMASK, bx + __popc(MX), 31);
    pt.ok = __all_sync(FULLMASK, bx + __popc(MX) <= TW && m0 + bn + __popc(MN) <= TW);
    if (pt.ok)
        warp_knots_stored<R, SPL, TW>(P, pt.v, lane * SPL, pt.km, pt.MX, pt.MN, pt.bx, pt.bn,
                                      pt.m0, pt.m1);
}

// ---------------------------------------------------------------------------------
// One sifting pass over one warp tile (the body of k_pass).
// STAGE: the next tile's inputs are copied into the stage buffer while this one computes
// (else only prefetched into L2: a smaller kernel, for launches with one tile per warp).
// `staged`: this tile's inputs are in the stage buffer (copied by the previous tile);
// `pre`: the inputs read before the kernel's wait (a warp's first tile), or null.
// Returns whether the next tile's were started.
template <typename R, int SPL, bool STAGE>
__device__ __forceinline__ bool pass_tile(const PassArgs &pa, WarpPool<R, 32 * SPL> &P,
                                          StageBuf<R, 32 * SPL> &B, int64_t gt, bool first,
                                          bool prefetch_next, bool staged,
                                          const PreTile<R, SPL> *pre)
{
    constexpr int TW = 32 * SPL;
    const int lane = threadIdx.x & 31;
    const int eh = lane >> 4, hl = lane & 15; // half-warp = envelope in the spline phases
    const int ii = pa.tile_inst[gt];
    State *stp = pa.state + ii;
    const Inst &in = pa.inst[ii];
    const int lt = (int)(gt - in.tile0);
    // the tile's interface values (written by the interface solve just before), read
    // together with the state unless the previous tile staged them
    SolveVals<R> sv{};
    int2 tpn = make_int2(0, 0);
    if (!(STAGE && staged)) {
        const TileSolve &so = in.tsol[(int64_t)eh * in.ntiles + lt];
        sv = solve_vals(so, R(0));
        tpn = *reinterpret_cast<const int2 *>(&so.tp);
    }
    const int mode = stp->mode;
    if (mode == MODE_DONE)
        return false;
    const int hpar = stp->hpar, rpar = stp->rpar, imfc = stp->imf_count;
    const int L = (int)in.L;
    if (lt == 0 && lane == 0) {
        stp->pass_mode = mode;
        stp->pass_sift = stp->sift_count;
        stp->pass_imf = imfc;
        stp->pass_par = hpar | (rpar << 1);
        stp->pass_scount = stp->scount;
    }
    const int ts = lt * TW;
    const int cnt = min(TW, L - ts);
    const bool hasL = ts > 0, hasR = ts + TW < L;
    const R *hsrc = (const R *)in.h[hpar] + ts;
    R *hdst = (R *)in.h[hpar ^ 1] + ts;
    const double *rsrc = in.r[rpar] + ts;
    double *rdst = in.r[rpar ^ 1] + ts;
    const bool sift = mode == MODE_SIFT || mode == MODE_SIFT_COMMIT;
    const bool commit = mode == MODE_SIFT_COMMIT || mode == MODE_COMMIT;
    const bool use_r = commit || mode == MODE_INIT;
    const int k0 = lane * SPL;

    R v[SPL], hn[SPL];
    R hcl = R(0), hcr = R(0); // current signal at the halo samples -1 and TW
    uint2 km = make_uint2(0u, 0u); // the signal's extremum masks and ranks (sifting modes)
    bool have = false;             // this tile's signal and knots came from `pre`
    if (STAGE && staged) {
        // copied in while the previous tile computed
        cp_async_wait_all();
        __syncwarp();
        vload<SPL>(B.stage + k0, v);
        if (lane == 0 && hasL)
            hcl = B.stage[TW];
        if (lane == 31 && hasR)
            hcr = B.stage[TW + 1];
        if (sift) {
            sv = solve_vals(B.sts[eh], R(0));
            tpn = *reinterpret_cast<const int2 *>(&B.sts[eh].tp);
            km = B.km[lane];
        }
        __syncwarp(); // the stage is refilled below
    } else {
        have = pre != nullptr && pre->hpar == hpar;
        if (mode != MODE_INIT) {
            if (have) {
#pragma unroll
                for (int s = 0; s < SPL; ++s)
                    v[s] = pre->v[s];
                hcl = pre->hcl;
                hcr = pre->hcr;
            } else {
                loadn<R, SPL>(hsrc, k0, cnt, v);
                if (lane == 0 && hasL)
                    hcl = hsrc[-1];
                if (lane == 31 && hasR)
                    hcr = hsrc[TW];
            }
        }
        if (sift)
            km = have ? pre->km : in.kmask[(int64_t)lt * 32 + lane];
    }
    // the warp's next tile: its signal and interface values into the stage buffer (or
    // its signal into L2), its residue (commit and INIT passes) into L2, while this one
    // computes
    bool nstaged = false;
    if constexpr (STAGE) {
        if (prefetch_next) {
            if (lt + 1 < in.ntiles) { // the same instance and mode: no descriptor reads
                if (mode != MODE_INIT) {
                    stage_issue<R, SPL>(B, mode, hsrc + TW, ts + TW, L, in.tsol, in.kmask,
                                        in.ntiles, lt + 1);
                    nstaged = true;
                }
            } else {
                nstaged = stage_tile<R, SPL>(pa, B, gt + 1);
            }
        }
    }
    // the residue of a commit (or INIT) pass into L2 now (a warp's first tile; the others
    // were prefetched by its previous tile), into registers when the sift is done
    if (first && use_r && lane == 0)
        prefetch_l2(rsrc, (uint32_t)(((cnt * 8) + 15) & ~15));
    if (prefetch_next && lane == 0 && lt + 1 < in.ntiles) {
        const int ncnt = min(TW, L - ts - TW);
        if (!STAGE && mode != MODE_INIT)
            prefetch_l2(hsrc + TW, (uint32_t)(((ncnt * (int)sizeof(R)) + 15) & ~15));
        if (use_r)
            prefetch_l2(rsrc + TW, (uint32_t)(((ncnt * 8) + 15) & ~15));
    }

    R pn = R(0), pd = R(0);
    int zc = 0;             // zero crossings of the sifted signal (S-number rule)
    R hnl = hcl, hnr = hcr; // the new signal at the halo samples
    if (sift) {
        // Step 1: the extrema of h were found when the previous pass wrote it (its masks
        // and ranks, stored per lane); only the knots are gathered into the pool
        uint32_t MX, MN;
        int bx, bn, m0, m1;
        if (have && pre->ok) { // compacted before the kernel's wait
            MX = pre->MX;
            MN = pre->MN;
            bx = pre->bx;
            bn = pre->bn;
            m0 = pre->m0;
            m1 = pre->m1;
        } else {
            warp_knots_stored<R, SPL, TW>(P, v, k0, km, MX, MN, bx, bn, m0, m1);
        }
        const int b1 = m0 + 2;
        const int base = eh ? b1 : 0, m = eh ? m1 : m0;
        if (hl == 0) {
            P.ky[base] = KnotY<R>{tpn.x - ts, sv.yp};
            P.ky[base + m + 1] = KnotY<R>{tpn.y - ts, sv.yn};
        }
        __syncwarp();
        env_solve_any<R, TW>(P, base, m, hl, m0, m1, sv);
        __syncwarp();
        // Steps 2-4 at every sample: both envelopes (interval = knots at or before k),
        // their mean, the subtraction, and the SD partial sums. A lane's samples share
        // few intervals: an interval's cubic is read when a knot starts it, and the local
        // coordinate u = k - t_left advances by exact integer steps in between.
        // The local coordinate of each sample is converted from the integer k - t, so the
        // samples' evaluations do not depend on one another (a short latency chain).
        int q0 = bx + (MX & 1u), q1 = b1 + bn + (MN & 1u);
        Coef<R> c0 = P.cf[q0], c1 = P.cf[q1];
        int t0 = P.ky[q0].t, t1 = P.ky[q1].t;
#pragma unroll
        for (int s = 0; s < SPL; ++s) {
            const int k = k0 + s;
            if (s > 0) {
                if ((MX >> s) & 1u) { // the knot is the sample itself
                    ++q0;
                    c0 = P.cf[q0];
                    t0 = k;
                }
                if ((MN >> s) & 1u) {
                    ++q1;
                    c1 = P.cf[q1];
                    t1 = k;
                }
            }
            const R e0 = horner(c0, R(k - t0));
            const R e1 = horner(c1, R(k - t1));
            const R mean = radd(e0, e1);
            hn[s] = rsub(v[s], mean);
            if (pa.need_sd && k < cnt) {
                pn += mean * mean;
                pd += v[s] * v[s];
            }
        }
        // the instance's last sample when it is a knot (the end-point rule puts one there,
        // as the right bracket of both envelopes): the envelopes take the knot values there
        // exactly, as at every other knot, instead of the cubic evaluated at the far end of
        // its interval; the loop left this lane's last intervals in c0 / c1
        if (!hasR && cnt - 1 >= k0 && cnt - 1 < k0 + SPL) {
            const KnotY<R> a0 = P.ky[m0 + 1], a1 = P.ky[b1 + m1 + 1];
            if (a0.t == cnt - 1 || a1.t == cnt - 1) {
                const R e0 = a0.t == cnt - 1 ? rmul(a0.y, R(0.5)) : horner(c0, R(cnt - 1 - t0));
                const R e1 = a1.t == cnt - 1 ? rmul(a1.y, R(0.5)) : horner(c1, R(cnt - 1 - t1));
#pragma unroll
                for (int s = 0; s < SPL; ++s)
                    if (k0 + s == cnt - 1)
                        hn[s] = rsub(v[s], radd(e0, e1));
            }
        }
        // halo samples: interval 0 before the tile, interval m after it (where the
        // bracket knot is the sample itself, the knot value, as the neighbour computes it)
        if (lane == 0 && hasL) {
            const R mean = radd(horner(P.cf[0], R(-1 - P.ky[0].t)),
                                horner(P.cf[b1], R(-1 - P.ky[b1].t)));
            hnl = rsub(hcl, mean);
        }
        if (lane == 31 && hasR) {
            const KnotY<R> a0 = P.ky[m0 + 1];
            const R e0 = a0.t == TW ? rmul(a0.y, R(0.5)) : horner(P.cf[m0], R(TW - P.ky[m0].t));
            const int q = b1 + m1;
            const KnotY<R> a1 = P.ky[q + 1];
            const R e1 = a1.t == TW ? rmul(a1.y, R(0.5)) : horner(P.cf[q], R(TW - P.ky[q].t));
            hnr = rsub(hcr, radd(e0, e1));
        }
        if (pa.need_zc) {
            // sign changes (negative vs not) between samples k and k+1 with k+1 in the tile;
            // the pair across the left tile edge uses the halo value, which equals the
            // neighbour's own result bit for bit
            const R nx = __shfl_down_sync(FULLMASK, hn[0], 1);
            int z = 0;
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const R b = s + 1 < SPL ? hn[s + 1] : nx;
                if (k0 + s + 1 < cnt && (lane < 31 || s + 1 < SPL))
                    z += ((hn[s] < R(0)) != (b < R(0))) ? 1 : 0;
            }
            if (lane == 0 && hasL)
                z += ((hnl < R(0)) != (hn[0] < R(0))) ? 1 : 0;
            zc = warp_sum(z);
        }
        __syncwarp(); // the pool is reused for the new signal's knots
    } else {
#pragma unroll
        for (int s = 0; s < SPL; ++s)
            hn[s] = v[s];
    }

    // Step 5 / Eq. (1): commit the IMF c, update the FP64 residue, restart from it (the
    // conversions between the working precision and FP64 run on the integer pipes)
    if (use_r) {
        double r[SPL], rl = 0.0, rr = 0.0;
        loadn<double, SPL>(rsrc, k0, cnt, r);
        if (lane == 0 && hasL)
            rl = rsrc[-1];
        if (lane == 31 && hasR)
            rr = rsrc[TW];
        if (commit) {
            double rn[SPL];
#pragma unroll
            for (int s = 0; s < SPL; ++s)
                rn[s] = __dsub_rn(r[s], widen(hn[s]));
            storen<double, SPL>(rdst, k0, cnt, rn);
            R *imf = (R *)in.imf + (int64_t)imfc * in.imf_stride;
            if (in.imf_serialized) {
                storen<R, SPL>(imf + ts, k0, cnt, hn);
            } else {
                const int64_t MD = in.M + in.D;
                const int p0 = ts + k0;
                int64_t i = p0 / MD, mm = p0 - i * MD;
#pragma unroll
                for (int s = 0; s < SPL; ++s) {
                    if (k0 + s < cnt && mm < in.M)
                        imf[in.order == 0 ? i * in.M + mm : mm * in.N + i] = hn[s];
                    if (++mm == MD) {
                        mm = 0;
                        ++i;
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < SPL; ++s)
                narrow_to(rn[s], hn[s]);
        } else {
#pragma unroll
            for (int s = 0; s < SPL; ++s)
                narrow_to(r[s], hn[s]);
        }
        if (lane == 0 && hasL)
            narrow_to(commit ? __dsub_rn(rl, widen(hnl)) : rl, hnl);
        if (lane == 31 && hasR)
            narrow_to(commit ? __dsub_rn(rr, widen(hnr)) : rr, hnr);
    }

    // Step 1 on the new signal and the per-tile elimination of its spline system
    {
        R left = __shfl_up_sync(FULLMASK, hn[SPL - 1], 1);
        R right = __shfl_down_sync(FULLMASK, hn[0], 1);
        if (lane == 0)
            left = hnl;
        if (lane == 31)
            right = hnr;
        uint32_t MX, MN;
        int bx, bn, m0, m1;
        warp_knots<R, SPL, TW>(P, hn, left, right, k0, ts + k0, cnt, L, MX, MN, bx, bn, m0, m1);
        // the masks and ranks for the next pass, which sifts this signal
        in.kmask[(int64_t)lt * 32 + lane] =
            make_uint2(MX | (MN << 16), (uint32_t)bx | ((uint32_t)bn << 16));
        __syncwarp();
        const int base = eh ? m0 + 2 : 0, m = eh ? m1 : m0;
        R f[3] = {R(0), R(0), R(0)}, l[3] = {R(0), R(0), R(0)};
        if (max(m0, m1) > kSparseKnots)
            env_export_any<R, TW>(P, base, m, hl, m0, m1, f, l);
        if (hl == 0) {
            TileRec<R> rec;
            rec.n = m;
            const int ix[4] = {0, min(1, m - 1), max(m - 2, 0), m - 1};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const KnotY<R> kq = P.ky[base + 1 + ix[q]];
                rec.t[q] = m >= 1 ? ts + kq.t : 0;
                rec.y[q] = m >= 1 ? kq.y : R(0);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                rec.xa[q] = m > kSparseKnots ? f[q] : R(0);
                rec.xb[q] = m > kSparseKnots ? l[q] : R(0);
            }
            store_rec(reinterpret_cast<TileRec<R> *>(in.tex) + (int64_t)eh * in.ntiles + lt, rec);
        }
        __syncwarp(); // the pool is reused by the warp's next tile
    }
    storen<R, SPL>(hdst, k0, cnt, hn);
    if (lane == 0 && !hasL)
        in.taux[lt].h_first = (double)hn[0];
    if (!hasR && k0 <= cnt - 1 && cnt - 1 < k0 + SPL) {
#pragma unroll
        for (int s = 0; s < SPL; ++s)
            if (k0 + s == cnt - 1)
                in.taux[lt].h_last = (double)hn[s];
    }
    if (sift && pa.need_sd) {
        pn = warp_sum(pn);
        pd = warp_sum(pd);
        if (lane == 0) {
            in.taux[lt].sd_num = (double)pn;
            in.taux[lt].sd_den = (double)pd;
        }
    }
    if (sift && pa.need_zc && lane == 0)
        in.taux[lt].nzc = zc;
    return nstaged;
}

// One sifting pass over all tiles of every running instance. Persistent grid: warp w
// takes the contiguous tile range [w C, w C + C) of the launch (C = tiles / warps,
// rounded up), so its next tile is usually the next tile of the same instance, which
// it prefetches into L2. Warps are independent (no block barrier).
// MINB is the register budget's target: the compiler keeps to the registers that let MINB
// CTAs reside on an SM (1: no limit). STAGE: see pass_tile.
template <typename R, int SPL, int NWARP, int MINB, bool STAGE>
__global__ void __launch_bounds__(NWARP * 32, MINB) k_pass(PassArgs pa)
{
    constexpr int TW = 32 * SPL;
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_trigger();
    const int warp = threadIdx.x >> 5;
    WarpPool<R, TW> &P = reinterpret_cast<WarpPool<R, TW> *>(smraw)[warp];
    // staging kernels: the stage buffers follow the NWARP pools (not touched otherwise)
    StageBuf<R, TW> &B =
        reinterpret_cast<StageBuf<R, TW> *>(smraw + NWARP * sizeof(WarpPool<R, TW>))[warp];
    const int64_t nw = (int64_t)gridDim.x * NWARP;
    const int64_t wid = (int64_t)blockIdx.x * NWARP + warp;
    const int64_t C = (pa.ntiles + nw - 1) / nw;
    const int64_t g0 = wid * C, g1 = min(g0 + C, pa.ntiles);
    // The tile -> instance map and the instance descriptors are written only before a
    // decomposition starts (host copies, or kernels that finished before the previous
    // kernel of the stream began), never by the pass or the interface solve: bring the
    // first tile's descriptor into L1 while the interface solve finishes. Nothing the
    // interface solve writes is touched before pdl_wait.
    if (g0 < g1 && (threadIdx.x & 31) < 2) {
        const char *d = reinterpret_cast<const char *>(pa.inst + pa.tile_inst[g0]);
        prefetch_l1(d + (threadIdx.x & 31) * (sizeof(Inst) - 1));
        if ((threadIdx.x & 31) == 0 && sizeof(Inst) > 128)
            prefetch_l1(d + 128);
    }
    // latency kernels: the first tile's signal while the interface solve finishes (the
    // staging kernels, with many tiles per warp, keep the registers for the tiles)
    PreTile<R, SPL> pre;
    if (!STAGE && g0 < g1)
        pre_tile<R, SPL>(pa, g0, pre, P);
    pdl_wait();
    bool staged = false;
    for (int64_t gt = g0; gt < g1; ++gt)
        staged = pass_tile<R, SPL, STAGE>(pa, P, B, gt, gt == g0, gt + 1 < g1, staged,
                                          (!STAGE && gt == g0) ? &pre : nullptr);
}


// ---------------------------------------------------------------------------------
// Interface solve: one CTA per instance and envelope (blockIdx.x = 2 instance +
// envelope). Both CTAs of an instance take the stop test and state-machine step from
// the same inputs (the pass's snapshot in State and the knot counts of both envelopes);
// the maxima CTA writes the state. Then the envelope's reduced interface system.
//
// Rows of the reduced system are the tile-edge knots in order, [mirrored or end knots]
// [first/last knot of every non-empty tile][mirrored or end knots]; a tile's interior
// knots next to its first/last knot are substituted by the tile's elimination
// (M = x0 + x1 M_first + x2 M_last), which keeps the system tridiagonal. The tile
// records are read once into a shared (or, for very long instances, global) scratch;
// every row is then built from the scratch alone. The solve has three levels in one
// warp: lane l eliminates its contiguous segment of rows in the working precision, the
// 32 segment-end unknowns are solved to FP64 accuracy, and the segments are
// back-substituted. GB300's FP64 pipe is narrow (a warp-wide FP64 instruction,
// conversions included, occupies it for many cycles), so FP32 plans keep FP64 out of the
// solve: the 32-unknown system is solved by FP32 cyclic reduction refined once with its
// residual evaluated in float-float arithmetic (FP64-accurate); FP64 plans run the
// cyclic reduction in FP64.

// Entry kinds of the reduced system.
enum EKind : int32_t {
    EK_FIXED = 0, // natural end: M = 0
    EK_FREE = 1,  // mirrored knot: plain row
    EK_F = 2,     // first knot of a tile with 2 knots (its right neighbour is the next entry)
    EK_FS = 3,    // first knot of a tile with >= 3 knots (right neighbour substituted)
    EK_L = 4,     // last knot of a tile with 2 knots
    EK_LS = 5,    // last knot of a tile with >= 3 knots (left neighbour substituted)
    EK_FL = 6     // the only knot of a tile
};

// Per-envelope scratch of k_reduce, structure of arrays of `cap` entries.
//   Et, Ey   - entry position and value
//   Ek       - entry kind
//   St, A..D - substituted neighbour (position St, value A) and the tile's elimination
//              (B, C, D = x0, x1, x2); then the row (a, b, c, d); then, for the rows a
//              segment eliminates, (bp, b, cp, dp)
//   MV       - solved second derivative
//   To       - per tile: the index of its first entry
//   Tu       - per tile: its number of entries (0, 1 or 2)
template <typename R>
struct RedScratch {
    R *Ey, *A, *B, *C, *D, *MV;
    int *Et, *Ek, *St, *To;
    unsigned char *Tu;
    __device__ void carve(unsigned char *p, int64_t cap)
    {
        R *r = reinterpret_cast<R *>(p);
        Ey = r;
        A = r + cap;
        B = r + 2 * cap;
        C = r + 3 * cap;
        D = r + 4 * cap;
        MV = r + 5 * cap;
        int *q = reinterpret_cast<int *>(r + 6 * cap);
        Et = q;
        Ek = q + cap;
        St = q + 2 * cap;
        To = q + 3 * cap;
        Tu = reinterpret_cast<unsigned char *>(q + 4 * cap);
    }
};

// Segment elimination of rows [rs, re) of the reduced system in the scratch, in place:
// rows rs..re-2 become (bp, b, cp, dp) in (A, B, C, D); returns the segment's reduced
// form (first unknown in terms of x_{rs-1} and x_{re-1}, last row kept). The scratch
// arrays are disjoint (__restrict__), so the loads of later rows may be issued ahead of
// the stores of earlier ones.
template <typename R>
__device__ __forceinline__ SegElim<R> seg_eliminate_rows(R *__restrict__ XA,
                                                         const R *__restrict__ XB,
                                                         R *__restrict__ XC, R *__restrict__ XD,
                                                         int rs, int re)
{
    SegElim<R> g;
    if (re - rs < 1)
        return g;
    R cprev = R(0), dprev = R(0), bprev = R(1);
    // the next row is loaded while the current one is eliminated (the loads do not wait
    // for the chain of reciprocals)
    R A = XA[rs], B = XB[rs], C = XC[rs], D = XD[rs];
#pragma unroll 2
    for (int j = rs; j < re - 1; ++j) {
        const R An = XA[j + 1], Bn = XB[j + 1], Cn = XC[j + 1], Dn = XD[j + 1];
        const R inv = rrcp(B - A * cprev);
        cprev = C * inv;
        dprev = (D - A * dprev) * inv;
        bprev = -A * bprev * inv;
        XA[j] = bprev;
        XC[j] = cprev;
        XD[j] = dprev;
        A = An;
        B = Bn;
        C = Cn;
        D = Dn;
    }
    g.al = A; // row re - 1, kept
    g.bl = B;
    g.cl = C;
    g.dl = D;
    if (re - rs >= 2) {
        g.alE = dprev;
        g.beE = bprev;
        g.gaE = -cprev;
        R xa = g.alE, xb = g.beE, xg = g.gaE;
#pragma unroll 4
        for (int j = re - 3; j >= rs; --j) {
            const R c = XC[j];
            xa = XD[j] - c * xa;
            xb = XA[j] - c * xb;
            xg = -c * xg;
        }
        g.alS = xa;
        g.beS = xb;
        g.gaS = xg;
    }
    return g;
}
template <typename R>
__device__ __forceinline__ SegElim<R> seg_eliminate(const RedScratch<R> &X, int rs, int re)
{
    return seg_eliminate_rows<R>(X.A, X.B, X.C, X.D, rs, re);
}

// Back-substitution of segment [rs, re) given x_{rs-1} = Zp and x_{re-1} = z; writes MV.
template <typename R>
__device__ __forceinline__ void seg_backsub_rows(const R *__restrict__ XA,
                                                 const R *__restrict__ XC,
                                                 const R *__restrict__ XD, R *__restrict__ XMV,
                                                 int rs, int re, R Zp, R z)
{
    if (re - rs < 1)
        return;
    XMV[re - 1] = z;
    R xn = z;
#pragma unroll 4
    for (int j = re - 2; j >= rs; --j) {
        const R x = XD[j] + XA[j] * Zp - XC[j] * xn;
        XMV[j] = x;
        xn = x;
    }
}
template <typename R>
__device__ __forceinline__ void seg_backsub(const RedScratch<R> &X, int rs, int re, R Zp, R z)
{
    seg_backsub_rows<R>(X.A, X.C, X.D, X.MV, rs, re, Zp, z);
}

struct RedCommon {
    double sd[kRedThreads / 32][2];
    int wsu[kRedThreads / 32], wsn[kRedThreads / 32][2], wzc[kRedThreads / 32];
    unsigned long long wpk[kRedThreads / 32];
    int next;
    double nakx[2][3]; // not-a-knot ends: the elimination data of rows 1 and NR - 2
};
// The large form's level-1 and level-1.5 arrays exist only in the kernel that has it.
template <bool SMALL>
struct RedShared : RedCommon {
    double lev[14 * kRedThreads]; // level-1 results (10 arrays), level-1.5 scratch (4), in R
    int segq[kRedThreads];        // rows per level-1 segment
};
template <>
struct RedShared<true> : RedCommon {
};
// Systems of at most this many rows are solved by warp 0 alone (three levels).
constexpr int kRedSmallRows = 24 * 32;

// Level 2: the 32 segment-end unknowns (one reduced row per lane, no outside values: the
// first and last rows are natural ends). FP64 plans: cyclic reduction in FP64.
__device__ __forceinline__ double level2_solve(const SegElim<double> &g, int q, bool has_next)
{
    const double zl[1] = {0.0}, zr[1] = {0.0};
    double Z[1];
    warp_reduced_solve<double, 1, 32>(g, q, has_next, zl, zr, Z);
    return Z[0];
}
// Error-free transformations of single-precision arithmetic (Dekker, Knuth): a product
// and a sum as an unevaluated pair hi + lo equal to the exact result.
__device__ __forceinline__ float two_prod(float a, float b, float &lo)
{
    const float p = __fmul_rn(a, b);
    lo = __fmaf_rn(a, b, -p);
    return p;
}
__device__ __forceinline__ float two_sum(float a, float b, float &lo)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
// A running sum in float-float (hi + lo, about 48 significant bits).
struct FFSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float h, float l)
    {
        float e;
        const float s = two_sum(hi, h, e);
        lo = __fadd_rn(__fadd_rn(lo, l), e);
        hi = s;
    }
    // a * b * c with the two products error-free (the last one's error to first order)
    __device__ __forceinline__ void add_prod3(float a, float b, float c)
    {
        float l1, l2;
        const float p1 = two_prod(a, b, l1);
        const float p2 = two_prod(p1, c, l2);
        add(p2, __fmaf_rn(l1, c, l2));
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
};

// FP32 plans: cyclic reduction in FP32, then the residual of the reduced rows evaluated in
// float-float arithmetic (error-free products and sums: about 48 significant bits, no FP64
// instruction, which GB300's narrow FP64 pipe would serialize) and one FP32 correction
// solve: the FP64-accurate solution of the system (it is diagonally dominant, condition
// number a few units). The reduced row of a lane (reduced_row) is expanded in the
// residual's terms: D - A z_{l-1} - B z_l - C z_{l+1} with A = al beE, B = bl + al gaE +
// cl nbeS, C = cl ngaS, D = dl - al alE - cl nalS.
__device__ __forceinline__ double level2_solve(const SegElim<float> &g, int q, bool has_next)
{
    const int lane = threadIdx.x & 31;
    const float nalS = __shfl_down_sync(FULLMASK, g.alS, 1);
    const float nbeS = __shfl_down_sync(FULLMASK, g.beS, 1);
    const float ngaS = __shfl_down_sync(FULLMASK, g.gaS, 1);
    float A, B, C, D;
    reduced_row(g, q, has_next, nalS, nbeS, ngaS, A, B, C, D);
    PcrFactors<float, 32> f;
    const float Z = pcr_solve_keep<float, 32>(A, B, C, D, f);
    float zm = __shfl_up_sync(FULLMASK, Z, 1), zp = __shfl_down_sync(FULLMASK, Z, 1);
    if (lane == 0)
        zm = 0.f;
    if (lane == 31)
        zp = 0.f;
    FFSum r;
    if (q >= 1) {
        r.add(g.dl, 0.f);
        r.add_prod3(-g.al, g.alE, 1.f);
        r.add_prod3(-g.al, g.beE, zm);
        r.add_prod3(-g.bl, 1.f, Z);
        r.add_prod3(-g.al, g.gaE, Z);
        if (has_next) {
            r.add_prod3(-g.cl, nalS, 1.f);
            r.add_prod3(-g.cl, nbeS, Z);
            r.add_prod3(-g.cl, ngaS, zp);
        }
    } else { // the dummy row Z = 0
        r.add_prod3(-1.f, 1.f, Z);
    }
    const float dZ = pcr_apply<float, 32>(f, r.value());
    return (double)Z + (double)dZ;
}

// The pass's snapshot of an instance's state (written by the pass kernel's first tile).
struct PassSnap {
    int pm, psift, pimf, ppar, pscount;
};

// Sec. 2.1 Step 5 and the IMF state machine, from the totals of the pass that just ran
// (knots of envelope e and of the other one, the SD sums, the zero crossings): returns the
// next mode. With `write` (one thread per instance) it also records the state, counts the
// instance as running and adds the pass's algorithmic bytes to the statistics.
template <typename R>
__device__ __forceinline__ int stop_step(const ReduceArgs &ra, const Inst &in, State *st,
                                         bool write, int e, int ntot, int nother, double sdn,
                                         double sdd, int nz, const PassSnap &ps)
{
    const int pm = ps.pm;
    const int nmax = e == 0 ? ntot : nother, nmin = e == 0 ? nother : ntot;
    const bool ok = nmax >= 1 && nmin >= 1 && nmax + nmin >= 3;
    int imf_count = ps.pimf, sift_count = ps.psift, scount = ps.pscount, nm;
    int committed = -1; // IMF slot whose sift count is recorded
    double sd = 0.0;
    if (pm == MODE_INIT || pm == MODE_COMMIT || pm == MODE_SIFT_COMMIT) {
        if (pm != MODE_INIT) {
            committed = imf_count;
            imf_count += 1;
        }
        if (imf_count >= ra.K || !ok) {
            nm = MODE_DONE;
        } else {
            nm = (ra.stop == STOP_FIXED && ra.fixed_sifts == 1) ? MODE_SIFT_COMMIT : MODE_SIFT;
        }
    } else {
        sift_count += 1;
        if (!ok) {
            nm = MODE_COMMIT;
        } else if (ra.stop == STOP_FIXED) {
            nm = (sift_count >= ra.fixed_sifts - 1) ? MODE_SIFT_COMMIT : MODE_SIFT;
        } else if (ra.stop == STOP_SD) {
            sd = sdn / sdd;
            nm = (sd < ra.sd_threshold || sift_count >= ra.max_sifts) ? MODE_COMMIT : MODE_SIFT;
        } else { // S-number: extrema and zero crossings of the sifted signal
            const int d = nmax + nmin - nz;
            scount = (d >= -1 && d <= 1) ? scount + 1 : 0;
            nm = (scount >= ra.s_number || sift_count >= ra.max_sifts) ? MODE_COMMIT : MODE_SIFT;
        }
    }
    if (write) {
        if (committed >= 0)
            st->sifts[committed] = sift_count + (pm == MODE_SIFT_COMMIT ? 1 : 0);
        if (pm == MODE_INIT || pm == MODE_COMMIT || pm == MODE_SIFT_COMMIT) {
            sift_count = 0;
            scount = 0;
        }
        st->scount = scount;
        st->hpar = (ps.ppar & 1) ^ 1;
        st->rpar = ((ps.ppar >> 1) & 1) ^ ((pm == MODE_SIFT_COMMIT || pm == MODE_COMMIT) ? 1 : 0);
        if (pm == MODE_SIFT && ra.stop == STOP_SD)
            st->sd = sd;
        st->imf_count = imf_count;
        st->sift_count = sift_count;
        st->nmax = nmax;
        st->nmin = nmin;
        st->mode = nm;
        if (nm != MODE_DONE)
            atomicAdd(ra.active, 1);
        if (ra.stats) {
            // algorithmic bytes per sample of the pass that just ran: h in (w) unless
            // INIT, h out (w), and for a commit the IMF out (w) and the residue in and
            // out (16); INIT reads the residue (8)
            const unsigned long long w = sizeof(R);
            unsigned long long per = (pm == MODE_INIT) ? 8 + w : 2 * w;
            if (pm == MODE_COMMIT || pm == MODE_SIFT_COMMIT)
                per += w + 16;
            atomicAdd(&ra.stats->pass_bytes, per * (unsigned long long)in.L);
            if (pm == MODE_SIFT || pm == MODE_SIFT_COMMIT)
                atomicAdd(&ra.stats->sample_sifts, (unsigned long long)in.L);
        }
    }
    return nm;
}

// SMALL: instances whose reduced systems have at most kRedSmallRows rows (the host
// guarantees it from the tile count); only the small form is compiled, with a register
// budget for three (FP32) or two (FP64) resident CTAs per SM instead of one or two, so
// that batches of many short instances fill the GPU (0: no register budget). NT: threads
// per CTA; the host launches NT = kRedThreadsTiny (with the same per-thread register
// budget, four times the CTAs per SM) when every instance has at most that many tiles.
// For such instances both thread counts perform the same operations in the same order
// (one tile per thread; the SD sums of warps past the tiles are exact zeros), so the
// results do not depend on which form ran.
template <typename R, bool SMALL, int NT = kRedThreads>
__global__ void __launch_bounds__(NT, SMALL ? (sizeof(R) == 4 ? 3 : 2) * (kRedThreads / NT) : 0)
    k_reduce(ReduceArgs ra)
{
    __shared__ RedShared<SMALL> S;
    const int e = blockIdx.x & 1;
    const int ii = ra.inst_list ? ra.inst_list[blockIdx.x >> 1] : (int)(blockIdx.x >> 1);
    // the instance descriptor does not change during a decomposition: read it while the
    // pass kernel finishes
    const Inst &in = ra.inst[ii];
    const int nt = in.ntiles;
    if (ra.cl > 0 && nt >= ra.cl_min_nt && nt <= ra.cl_max_nt)
        return; // the cluster kernel's instance
    const TileRec<R> *texe = reinterpret_cast<const TileRec<R> *>(in.tex) + (int64_t)e * nt;
    const TileRec<R> *texo = reinterpret_cast<const TileRec<R> *>(in.tex) + (int64_t)(e ^ 1) * nt;
    TileSolve *tsol = in.tsol + (int64_t)e * nt;
    const TileAux *taux = in.taux;
    RedScratch<R> X;
    {
        extern __shared__ __align__(16) unsigned char rsm[];
        const bool shm = ra.smem_entries > 0;
        const int64_t cap = shm ? ra.smem_entries : in.rlen;
        unsigned char *p0 = shm ? rsm
                                : reinterpret_cast<unsigned char *>(in.rscr + e * rscr_env_doubles(cap));
        X.carve(p0, cap);
    }
    pdl_wait();
    // the next pass may start now: the pass this solve waited for is complete, so the next
    // one can read that pass's signal before its own wait
    pdl_trigger();
    // what the pass kernel wrote is read at once (the state and the tile counts; the
    // counts of a finished instance are read and dropped)
    State *st = ra.state + ii;
    const int mode_now = st->mode;
    const int pm = st->pass_mode, psift = st->pass_sift, pimf = st->pass_imf;
    const int ppar = st->pass_par, pscount = st->pass_scount;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NW = NT / 32;

    // counts: knots of both envelopes, this envelope's reduced-system entries per tile
    // (first/last knot) and the SD sums of the pass that just ran. With at most one tile
    // per thread, the thread loads its tile's whole record here and writes the tile's
    // entries from registers once the offsets are known; the offsets and totals come from
    // one block scan of (entries, knots, the other envelope's knots) packed in 64 bits
    // (12, 19 and 33 bits: at most 4 x 256 entries and 256 x 512 knots). Otherwise tiles
    // are taken in a stride of the block, four per thread at a time, every load in flight
    // before use, and each thread then writes the entries of a contiguous chunk of tiles.
    int sn = 0, so_ = 0, zs = 0;
    double a = 0.0, b = 0.0;
    const bool want_sd = ra.stop == STOP_SD, want_zc = ra.stop == STOP_SNUMBER;
    const bool one = nt <= NT;
    int ntot = 0, nother = 0, U = 0, ubase = 0, u1 = 0, ca = 0, cb = 0;
    TileRec<R> r1;
    r1.n = 0;
    if (one) {
        if (tid < nt) {
            r1 = load_rec(texe + tid);
            so_ = texo[tid].n;
            if (want_sd) {
                a = taux[tid].sd_num;
                b = taux[tid].sd_den;
            }
            if (want_zc)
                zs = taux[tid].nzc;
            sn = r1.n;
        }
        if (mode_now == MODE_DONE)
            return;
        u1 = sn <= kSparseKnots ? sn : 2;
        const uint64_t pk = (uint64_t)u1 | ((uint64_t)sn << 12) | ((uint64_t)so_ << 31);
        uint64_t incl = pk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(FULLMASK, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            S.wpk[warp] = incl;
        if (want_zc) {
            zs = warp_sum(zs);
            if (lane == 0)
                S.wzc[warp] = zs;
        }
        if (want_sd) { // FP64 sums only when the stop rule reads them (the FP64 pipe is narrow)
            a = warp_sum(a);
            b = warp_sum(b);
            if (lane == 0) {
                S.sd[warp][0] = a;
                S.sd[warp][1] = b;
            }
        }
        if (tid < nt)
            X.Tu[tid] = (unsigned char)u1;
        __syncthreads();
        uint64_t before = incl - pk, tot = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint64_t v = S.wpk[w];
            before += w < warp ? v : 0;
            tot += v;
        }
        ubase = (int)(before & 0xfffu);
        U = (int)(tot & 0xfffu);
        ntot = (int)((tot >> 12) & 0x7ffffu);
        nother = (int)(tot >> 31);
    } else {
        for (int t0 = 0; t0 < nt; t0 += 4 * NT) {
            int ne[4], no[4], nz[4];
            double sa[4], sb[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int t = t0 + tid + k * NT;
                ne[k] = no[k] = nz[k] = 0;
                sa[k] = sb[k] = 0.0;
                if (t < nt) {
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
                const int t = t0 + tid + k * NT;
                if (t < nt)
                    X.Tu[t] = (unsigned char)(ne[k] <= kSparseKnots ? ne[k] : 2);
                sn += ne[k];
                so_ += no[k];
                zs += nz[k];
                a += sa[k];
                b += sb[k];
            }
        }
        if (mode_now == MODE_DONE)
            return;
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
        // entry offsets: each thread sums a contiguous chunk of tiles, a block scan of the
        // chunk sums, then the chunk's per-tile offsets
        const int CH = (nt + NT - 1) / NT;
        ca = min(tid * CH, nt);
        cb = min(ca + CH, nt);
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
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            ntot += S.wsn[w][0];
            nother += S.wsn[w][1];
        }
        __syncthreads();
        ubase = incl - su;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            ubase += w < warp ? S.wsu[w] : 0;
            U += S.wsu[w];
        }
    }
    // the stop test and the next mode (a middle thread, while the others write the
    // entries: thread 0 also writes the mirrored end rows of the first tile; the entries
    // of an instance that stops sifting are dropped)
    if (tid == NT / 2) {
        double sdn = 0.0, sdd = 0.0;
        int nz = 0;
        for (int w = 0; w < NW; ++w) {
            if (want_sd) {
                sdn += S.sd[w][0];
                sdd += S.sd[w][1];
            }
            if (want_zc)
                nz += S.wzc[w];
        }
        const PassSnap ps{pm, psift, pimf, ppar, pscount};
        S.next = stop_step<R>(ra, in, st, e == 0, e, ntot, nother, sdn, sdd, nz, ps);
    }
    const int nl = ra.boundary == BND_MIRROR ? min(ra.mirror_knots, ntot) : 1;
    const int nr = nl;
    const int NR = nl + U + nr;
    // not-a-knot ends need a sequence of at least four knots (boundary knots included)
    const bool nak = ra.spline_end == SPLINE_NOT_A_KNOT && ntot + nl + nr >= 4;
    auto put_entries = [&](const TileRec<R> &rc, int p) {
        const int n = rc.n;
        if (n == 1) {
            X.Et[p] = rc.t[0];
            X.Ey[p] = rc.y[0];
            X.Ek[p] = EK_FL;
        } else if (n >= 2 && n <= kSparseKnots) {
            // every knot an entry: t[0], t[1] (n >= 3), t[2] (n = 4), t[3]
            X.Et[p] = rc.t[0];
            X.Ey[p] = rc.y[0];
            X.Ek[p] = EK_F;
            int q = p + 1;
            if (n >= 3) {
                X.Et[q] = rc.t[1];
                X.Ey[q] = rc.y[1];
                X.Ek[q] = EK_FREE;
                ++q;
            }
            if (n == 4) {
                X.Et[q] = rc.t[2];
                X.Ey[q] = rc.y[2];
                X.Ek[q] = EK_FREE;
                ++q;
            }
            X.Et[q] = rc.t[3];
            X.Ey[q] = rc.y[3];
            X.Ek[q] = EK_L;
        } else if (n > kSparseKnots) {
            X.Et[p] = rc.t[0];
            X.Ey[p] = rc.y[0];
            X.Et[p + 1] = rc.t[3];
            X.Ey[p + 1] = rc.y[3];
            {
                X.Ek[p] = EK_FS;
                X.St[p] = rc.t[1];
                X.A[p] = rc.y[1];
                X.B[p] = rc.xa[0];
                X.C[p] = rc.xa[1];
                X.D[p] = rc.xa[2];
                X.Ek[p + 1] = EK_LS;
                X.St[p + 1] = rc.t[2];
                X.A[p + 1] = rc.y[2];
                X.B[p + 1] = rc.xb[0];
                X.C[p + 1] = rc.xb[1];
                X.D[p + 1] = rc.xb[2];
            }
        }
    };
    if (one) {
        if (tid < nt) {
            X.To[tid] = nl + ubase;
            put_entries(r1, nl + ubase);
        }
        // the end knots, written beside the entries: mirrored knots by the threads that hold
        // the signal's first two and last two knots (a tile's first and second knots are
        // t[0], t[1], its second-to-last and last t[2], t[3]; a tile with one knot has
        // t[0] = t[3]); end samples by two threads of warp 1
        if (ra.boundary == BND_MIRROR) {
            if (tid < nt && u1 >= 1) {
                const int n = r1.n, l = nl + U - 1;
                const int Lm = (int)(2 * (in.L - 1));
                if (ubase == 0) {
                    X.Et[nl - 1] = -r1.t[0];
                    X.Ey[nl - 1] = r1.y[0];
                    X.Ek[nl - 1] = nl == 2 ? EK_FREE : EK_FIXED;
                    if (nl == 2 && n >= 2) {
                        X.Et[0] = -r1.t[1];
                        X.Ey[0] = r1.y[1];
                        X.Ek[0] = EK_FIXED;
                    }
                } else if (ubase == 1 && nl == 2) { // the first tile has one knot
                    X.Et[0] = -r1.t[0];
                    X.Ey[0] = r1.y[0];
                    X.Ek[0] = EK_FIXED;
                }
                if (ubase + u1 == U) {
                    X.Et[l + 1] = Lm - r1.t[3];
                    X.Ey[l + 1] = r1.y[3];
                    X.Ek[l + 1] = nr == 2 ? EK_FREE : EK_FIXED;
                    if (nr == 2 && n >= 2) {
                        X.Et[l + 2] = Lm - r1.t[2];
                        X.Ey[l + 2] = r1.y[2];
                        X.Ek[l + 2] = EK_FIXED;
                    }
                } else if (ubase + u1 == U - 1 && nr == 2) { // the last tile has one knot
                    X.Et[l + 2] = Lm - r1.t[3];
                    X.Ey[l + 2] = r1.y[3];
                    X.Ek[l + 2] = EK_FIXED;
                }
            }
        } else if (tid == 32) {
            X.Et[0] = 0;
            X.Ey[0] = (R)in.taux[0].h_first;
            X.Ek[0] = EK_FIXED;
        } else if (tid == 33) {
            X.Et[nl + U] = (int)(in.L - 1);
            X.Ey[nl + U] = (R)in.taux[nt - 1].h_last;
            X.Ek[nl + U] = EK_FIXED;
        }
    } else {
        {
            int p = nl + ubase;
            for (int t = ca; t < cb; ++t) {
                X.To[t] = p;
                p += X.Tu[t];
            }
        }
        __syncthreads();
        // entries, with the substitution data of their rows: tiles in a stride of the
        // block, four records per thread in flight at a time
        for (int t0 = 0; t0 < nt; t0 += 4 * NT) {
            TileRec<R> rb[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int t = t0 + tid + k * NT;
                if (t < nt)
                    rb[k] = load_rec(texe + t);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int t = t0 + tid + k * NT;
                if (t >= nt)
                    break;
                put_entries(rb[k], X.To[t]);
            }
        }
    }
    __syncthreads();
    const int nm = S.next;
    if (nm != MODE_SIFT && nm != MODE_SIFT_COMMIT)
        return;
    if (!one && tid == 0) {
        const int64_t L = in.L;
        if (ra.boundary == BND_MIRROR) {
            // first two and last two knots of the whole signal, reflected about the ends
            const int f = nl, l = nl + U - 1;
            if (nl == 2) {
                // the signal's second knot: substituted neighbour of a first knot, else
                // the next entry
                const bool sub = X.Ek[f] == EK_FS;
                const int t1 = sub ? X.St[f] : X.Et[f + 1];
                const R y1 = sub ? X.A[f] : X.Ey[f + 1];
                X.Et[0] = -t1;
                X.Ey[0] = y1;
                X.Ek[0] = EK_FIXED;
                X.Et[1] = -X.Et[f];
                X.Ey[1] = X.Ey[f];
                X.Ek[1] = EK_FREE;
            } else {
                X.Et[0] = -X.Et[f];
                X.Ey[0] = X.Ey[f];
                X.Ek[0] = EK_FIXED;
            }
            const int Lm = (int)(2 * (L - 1));
            if (nr == 2) {
                const bool sub = X.Ek[l] == EK_LS;
                const int t2 = sub ? X.St[l] : X.Et[l - 1];
                const R y2 = sub ? X.A[l] : X.Ey[l - 1];
                X.Et[l + 1] = Lm - X.Et[l];
                X.Ey[l + 1] = X.Ey[l];
                X.Ek[l + 1] = EK_FREE;
                X.Et[l + 2] = Lm - t2;
                X.Ey[l + 2] = y2;
                X.Ek[l + 2] = EK_FIXED;
            } else {
                X.Et[l + 1] = Lm - X.Et[l];
                X.Ey[l + 1] = X.Ey[l];
                X.Ek[l + 1] = EK_FIXED;
            }
        } else {
            X.Et[0] = 0;
            X.Ey[0] = (R)in.taux[0].h_first;
            X.Ek[0] = EK_FIXED;
            X.Et[nl + U] = (int)(L - 1);
            X.Ey[nl + U] = (R)in.taux[nt - 1].h_last;
            X.Ek[nl + U] = EK_FIXED;
        }
    }
    if (!one)
        __syncthreads();
    // rows, every thread a strided share (reads the scratch only; writes its own rows)
    for (int p = tid; p < NR; p += NT) {
        const int k = X.Ek[p];
        R ra_ = R(0), rb = R(1), rc_ = R(0), rd = R(0);
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
            R a = hl, b = R(2) * (hl + hr), c = hr;
            if (nak && p == 1) {
                // not-a-knot: M_0 = ((h_0 + h_1) M_1 - h_0 M_2) / h_1 substituted
                b = b + hl * (hl + hr) * rrcp(hr);
                c = hr - hl * hl * rrcp(hr);
                a = R(0);
                if (k == EK_FS) {
                    S.nakx[0][0] = (double)x0;
                    S.nakx[0][1] = (double)x1;
                    S.nakx[0][2] = (double)x2;
                }
            }
            if (nak && p == NR - 2) {
                // M_{n-1} = ((h_{n-3} + h_{n-2}) M_{n-2} - h_{n-2} M_{n-3}) / h_{n-3}
                b = b + hr * (hl + hr) * rrcp(hl);
                a = hl - hr * hr * rrcp(hl);
                c = R(0);
                if (k == EK_LS) {
                    S.nakx[1][0] = (double)x0;
                    S.nakx[1][1] = (double)x1;
                    S.nakx[1][2] = (double)x2;
                }
            }
            ra_ = a;
            rb = b;
            rc_ = c;
            rd = d0;
            if (k == EK_FS) {
                rb = b + c * x1;
                rc_ = c * x2;
                rd = d0 - c * x0;
            } else if (k == EK_LS) {
                rb = b + a * x2;
                ra_ = a * x1;
                rd = d0 - a * x0;
            }
        }
        X.A[p] = ra_;
        X.B[p] = rb;
        X.C[p] = rc_;
        X.D[p] = rd;
    }
    __syncthreads();
    // small systems: three levels in warp 0 (segments of Q1 rows per lane, the 32 segment
    // ends to FP64 accuracy, back-substitution)
    auto small_solve = [&]() {
        if (warp == 0) {
            const int Q1 = ((NR + 31) >> 5) | 1;
            const int rs = min(lane * Q1, NR), re = min(rs + Q1, NR), rq = re - rs;
            const SegElim<R> g = seg_eliminate(X, rs, re);
            const double Zd = level2_solve(g, rq, (rq >= 1) && (re < NR));
            const R z = (R)Zd;
            R Zp = __shfl_up_sync(FULLMASK, z, 1);
            if (lane == 0)
                Zp = R(0);
            seg_backsub(X, rs, re, Zp, z);
        }
        __syncthreads();
    };
    if constexpr (SMALL) {
        small_solve();
    } else if (NR <= kRedSmallRows) {
        small_solve();
    } else {
        R *lev = reinterpret_cast<R *>(S.lev);
        constexpr int NS = NT;     // level-1 segments of the large form
        constexpr int G = NT / 32; // segments per lane of the level-1.5 warp
        // transposed layout: lane l's k-th segment (j = G l + k) at k * 32 + l, so
        // that the level-1.5 warp reads without bank conflicts
        auto tj = [](int j) { return (j % G) * 32 + j / G; };
        // level 1: every thread eliminates a contiguous segment of Q1 rows (Q1 odd, so
        // the lanes of a warp hit distinct banks)
        const int Q1 = ((NR + NS - 1) / NS) | 1;
        const int rs = min(tid * Q1, NR), re = min(rs + Q1, NR), rq = re - rs;
        {
            const SegElim<R> g = seg_eliminate(X, rs, re);
            const R gv[10] = {g.alS, g.beS, g.gaS, g.alE, g.beE, g.gaE, g.al, g.bl, g.cl, g.dl};
#pragma unroll
            for (int k = 0; k < 10; ++k)
                lev[k * NS + tj(tid)] = gv[k];
            S.segq[tj(tid)] = rq;
        }
        __syncthreads();
        if (warp == 0) {
            // level 1.5: the NS segment-end unknowns; lane l eliminates the reduced rows of
            // segments G l .. G l + G - 1 (row j couples Z_{j-1}, Z_j, Z_{j+1})
            R *cp2 = lev + 10 * NS, *dp2 = lev + 11 * NS, *bp2 = lev + 12 * NS;
            R *Zs = lev + 13 * NS;
            auto red_row = [&](int k, R &A, R &B, R &C, R &D) {
                // reduced row of segment j = G lane + k; its successor is j + 1
                const int i = k * 32 + lane;
                SegElim<R> gj;
                gj.alE = lev[3 * NS + i];
                gj.beE = lev[4 * NS + i];
                gj.gaE = lev[5 * NS + i];
                gj.al = lev[6 * NS + i];
                gj.bl = lev[7 * NS + i];
                gj.cl = lev[8 * NS + i];
                gj.dl = lev[9 * NS + i];
                const int j = G * lane + k;
                const int in_ = j + 1 < NS ? tj(j + 1) : 0;
                const bool hn = j + 1 < NS && S.segq[in_] >= 1;
                const R nalS = hn ? lev[in_] : R(0), nbeS = hn ? lev[NS + in_] : R(0);
                const R ngaS = hn ? lev[2 * NS + in_] : R(0);
                reduced_row(gj, S.segq[i], hn, nalS, nbeS, ngaS, A, B, C, D);
            };
            SegElim<R> g2;
            R cprev = R(0), dprev = R(0), bprev = R(1);
#pragma unroll
            for (int k = 0; k < G - 1; ++k) {
                R A, B, C, D;
                red_row(k, A, B, C, D);
                const R inv = rrcp(B - A * cprev);
                cprev = C * inv;
                dprev = (D - A * dprev) * inv;
                bprev = -A * bprev * inv;
                cp2[k * 32 + lane] = cprev;
                dp2[k * 32 + lane] = dprev;
                bp2[k * 32 + lane] = bprev;
            }
            red_row(G - 1, g2.al, g2.bl, g2.cl, g2.dl);
            g2.alE = dprev;
            g2.beE = bprev;
            g2.gaE = -cprev;
            R xa = g2.alE, xb = g2.beE, xg = g2.gaE;
#pragma unroll
            for (int k = G - 3; k >= 0; --k) {
                const R c = cp2[k * 32 + lane];
                xa = dp2[k * 32 + lane] - c * xa;
                xb = bp2[k * 32 + lane] - c * xb;
                xg = -c * xg;
            }
            g2.alS = xa;
            g2.beS = xb;
            g2.gaS = xg;
            // level 2: the 32 group-end unknowns to FP64 accuracy
            const double Zd = level2_solve(g2, G, lane < 31);
            const R z = (R)Zd;
            R Zp = __shfl_up_sync(FULLMASK, z, 1);
            if (lane == 0)
                Zp = R(0);
            Zs[(G - 1) * 32 + lane] = z;
            R xn = z;
#pragma unroll
            for (int k = G - 2; k >= 0; --k) {
                const int i = k * 32 + lane;
                const R x = dp2[i] + bp2[i] * Zp - cp2[i] * xn;
                Zs[i] = x;
                xn = x;
            }
        }
        __syncthreads();
        // level 3: back-substitution of this thread's segment
        if (rq >= 1) {
            const R *Zs = lev + 13 * NS;
            seg_backsub(X, rs, re, tid > 0 ? Zs[tj(tid - 1)] : R(0), Zs[tj(tid)]);
        }
        __syncthreads();
    
    }
    if (nak) {
        // the end knots' second derivatives from the not-a-knot conditions (the solve
        // held them at 0); the third knot (second-to-last) may be a tile interior knot,
        // given by the tile's elimination
        if (tid == 0) {
            const bool sub = X.Ek[1] == EK_FS;
            const R h0 = R(X.Et[1] - X.Et[0]), h1 = R((sub ? X.St[1] : X.Et[2]) - X.Et[1]);
            const R M1 = X.MV[1];
            const R M2 = sub ? (R)S.nakx[0][0] + (R)S.nakx[0][1] * M1 + (R)S.nakx[0][2] * X.MV[2]
                             : X.MV[2];
            X.MV[0] = ((h0 + h1) * M1 - h0 * M2) * rrcp(h1);
        } else if (tid == 32) {
            const int q = NR - 2;
            const bool sub = X.Ek[q] == EK_LS;
            const R hb = R(X.Et[q + 1] - X.Et[q]), ha = R(X.Et[q] - (sub ? X.St[q] : X.Et[q - 1]));
            const R Mq = X.MV[q];
            const R M3 = sub ? (R)S.nakx[1][0] + (R)S.nakx[1][1] * X.MV[q - 1] + (R)S.nakx[1][2] * Mq
                             : X.MV[q - 1];
            X.MV[NR - 1] = ((ha + hb) * Mq - hb * M3) * rrcp(ha);
        }
        __syncthreads();
    }
    for (int t = tid; t < nt; t += NT) {
        const int u = X.Tu[t], p = X.To[t];
        TileSolve *so = tsol + t;
        const R yp = X.Ey[p - 1], Mp = X.MV[p - 1], yn = X.Ey[p + u], Mn = X.MV[p + u];
        const R MF = u >= 1 ? X.MV[p] : R(0), ML = u >= 1 ? X.MV[p + u - 1] : R(0);
        const R M1 = u >= 3 ? X.MV[p + 1] : R(0), M2 = u >= 4 ? X.MV[p + 2] : R(0);
        so->tp = X.Et[p - 1];
        so->tn = X.Et[p + u];
        if (sizeof(R) == 4) {
            // FP32 pass kernels read the single-precision values only
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
}

} // namespace semd
