// Device side of the GB300 Serial-EMD library: the sifting pass kernel, the interface
// solve of the partitioned spline system, and the warp-level tridiagonal machinery.
//
// Method (Zhang et al., arXiv 2106.15319): serialize the input (Sec. 3.2), sift the 1D
// signal (Sec. 2.1 Steps 1-5: extrema, cubic-spline envelopes, mean, subtract, stop
// test), commit IMFs (Eq. 1) and de-serialize (Sec. 3.3).
//
// Pass structure. Every instance's serialized signal is cut into tiles of TILE samples;
// one CTA owns one tile and each thread 8 consecutive samples. A pass reads the current
// signal h once and writes the next one once:
//   k_pass   (per tile)     - extrema of h as bit masks (Step 1), compaction of the knot
//                             positions, the tile's spline second derivatives given the
//                             tile-boundary values from the previous k_reduce, the
//                             interval cubics, envelope evaluation, mean and subtraction
//                             (Steps 2-4), SD partial sums, IMF commit (Step 5 / Eq. 1);
//                             then extrema of the new signal and elimination of the
//                             tile's interior knots (the per-chunk part of the
//                             partitioned spline solve), exported as a short record.
//   k_reduce (per instance) - assembles the reduced interface system (two unknowns per
//                             tile and envelope, plus the end knots), solves it in
//                             FP64, writes the tile-boundary values back, and runs the
//                             stop test / IMF state machine for the next pass.
// Knot lists never leave shared memory: besides the signal, only ~100 bytes per tile
// and envelope cross HBM.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "semd_types.h"

namespace semd {

// Skewed index for the interface solve's scratch (lanes walking contiguous segments hit
// distinct shared-memory banks).
__device__ __forceinline__ int sk(int j) { return j + (j >> 5); }

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
// Reciprocals: the hardware approximation in FP32 (about 2 ulp); in FP64 a float seed
// refined by two Newton steps (about 1 ulp), which avoids the long IEEE division
// sequence on the narrow FP64 pipe. Both are deterministic, which is what the halo
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

// ---------------------------------------------------------------------------------
// Warp-level partitioned tridiagonal solve.
//
// Unknowns x_0..x_{n-1}; row i: a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i, with the
// outside values x_{-1} = xl[col] and x_n = xr[col] given per right-hand-side column.
// Column 0 carries d; columns 1.. have d = 0 (they give the response to the outside
// values). Lane l owns rows [s, e); it eliminates rows s..e-2 with the Thomas algorithm
// in terms of x_{s-1} (last unknown of lane l-1) and x_{e-1} (its own last unknown
// Z_l), which leaves one reduced row per lane coupling Z_{l-1}, Z_l, Z_{l+1}. That
// 32-unknown system is solved by parallel cyclic reduction over shuffles. The matrix is
// diagonally dominant (spline rows: b = 2(a + c)), so no pivoting is needed.

// Per-lane result of the segment elimination: x_s = alS + beS x_{s-1} + gaS Z_l,
// x_{e-2} = alE + beE x_{s-1} + gaE Z_l, and the lane's last row (al, bl, cl, dl).
template <typename R>
struct SegElim {
    R alS = R(0), beS = R(0), gaS = R(1), alE = R(0), beE = R(1), gaE = R(0);
    R al = R(0), bl = R(1), cl = R(0), dl = R(0);
};

// The reduced 32-unknown system and its solution by parallel cyclic reduction; returns
// Z_l per column (dummy 0 for lanes without rows, q == 0).
template <typename R, int NCOL>
__device__ __forceinline__ void warp_reduced_solve(const SegElim<R> &g, int q, bool has_next,
                                                   const R (&xl)[NCOL], const R (&xr)[NCOL],
                                                   R (&Z)[NCOL])
{
    const int lane = threadIdx.x & 31;
    const R nalS = __shfl_down_sync(FULLMASK, g.alS, 1);
    const R nbeS = __shfl_down_sync(FULLMASK, g.beS, 1);
    const R ngaS = __shfl_down_sync(FULLMASK, g.gaS, 1);
    R A = R(0), B = R(1), C = R(0), D[NCOL];
#pragma unroll
    for (int k = 0; k < NCOL; ++k)
        D[k] = R(0);
    if (q >= 1) {
        A = g.al * g.beE;
        B = g.bl + g.al * g.gaE + (has_next ? g.cl * nbeS : R(0));
        C = has_next ? g.cl * ngaS : R(0);
        D[0] = g.dl - g.al * g.alE - (has_next ? g.cl * nalS : R(0));
        if (lane == 0) {
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
    const R invB = rrcp(B);
#pragma unroll
    for (int k = 0; k < NCOL; ++k)
        Z[k] = D[k] * invB;
}

// General form used by the interface solve: rows from a functor, per-row scratch
// cp/dp/bp (skewed index), full back-substitution through `out`.
template <typename R, class RowFn, class OutFn>
__device__ void warp_tridiag(int n, const RowFn &row, R xl0, R xr0, R *cp, R *dp, R *bp,
                             const OutFn &out)
{
    const int lane = threadIdx.x & 31;
    const int Q = (n + 31) >> 5;
    const int s = min(lane * Q, n), e = min(s + Q, n), q = e - s;
    SegElim<R> g;
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
        g.alE = dprev;
        g.beE = bprev;
        g.gaE = -cprev;
        R xa = g.alE, xb = g.beE, xg = g.gaE;
        for (int j = e - 3; j >= s; --j) {
            const R c = cp[sk(j)];
            xa = dp[sk(j)] - c * xa;
            xb = bp[sk(j)] - c * xb;
            xg = -c * xg;
        }
        g.alS = xa;
        g.beS = xb;
        g.gaS = xg;
    }
    if (q >= 1)
        row(e - 1, g.al, g.bl, g.cl, g.dl);
    const R xl[1] = {xl0}, xr[1] = {xr0};
    R Z[1];
    warp_reduced_solve<R, 1>(g, q, (q >= 1) && (e < n), xl, xr, Z);
    R Zp = __shfl_up_sync(FULLMASK, Z[0], 1);
    if (lane == 0)
        Zp = xl0;
    if (q >= 1) {
        out(e - 1, Z[0]);
        R xn = Z[0];
        for (int j = e - 2; j >= s; --j) {
            const R x = dp[sk(j)] + bp[sk(j)] * Zp - cp[sk(j)] * xn;
            out(j, x);
            xn = x;
        }
    }
}

// Rows of the reduced interface system, read from (shared or global) scratch.
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
// Shared memory of one tile pass.
//
// Per envelope: the knot positions (tile-relative), kte[0] = bracket knot before the
// tile, kte[j + 1] = knot j, kte[m + 1] = bracket knot after the tile; the interval
// cubics cf[q], q = 0..m (interval q runs from knot q-1 to knot q), which during the
// solve hold the interval's slope, 1/length, length and left value; per-row
// elimination scratch rw (cp, dp, bp). A lane of the solving warp walks a contiguous
// run of Q rows with Q odd, so the 32 lanes always touch distinct banks.
template <typename R, int TILE>
struct EnvSmem {
    static constexpr int KC = TILE / 2 + 2; // knots of one kind in a tile, with room
    Coef<R> cf[KC + 2];
    Coef<R> rw[KC];
    int kte[KC + 4];
};

template <typename R, int TILE, int NT>
struct PassSmem {
    static constexpr int NW = NT / 32;
    EnvSmem<R, TILE> env[2];
    R hs[TILE + 8];   // hs[4 + k]: signal at tile-relative k, k in [-1, TILE]
    uint32_t wcnt[NW];
    R red[2][NW];
    int cnt[2];
};

// The interface solution of one tile and envelope in the working precision (FP32 pass
// kernels read the single-precision copy, so they issue no FP64 conversions).
template <typename R>
struct SolveVals {
    R MF, ML, yp, Mp, yn, Mn;
};
__device__ __forceinline__ SolveVals<float> solve_vals(const TileSolve &so, float)
{
    return {so.f[0], so.f[1], so.f[2], so.f[3], so.f[4], so.f[5]};
}
__device__ __forceinline__ SolveVals<double> solve_vals(const TileSolve &so, double)
{
    return {so.MF, so.ML, so.yp, so.Mp, so.yn, so.Mn};
}

// Stores v in an 8-byte record slot: as a double, or as a float in the slot's first half.
__device__ __forceinline__ void put_slot(double *slot, double v) { *slot = v; }
__device__ __forceinline__ void put_slot(double *slot, float v)
{
    *reinterpret_cast<float *>(slot) = v;
}

template <typename R>
struct Vec8;
template <>
struct Vec8<float> {
    __device__ static void load(const float *p, float (&v)[8])
    {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        const float4 b = *reinterpret_cast<const float4 *>(p + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    __device__ static void store(float *p, const float (&v)[8])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
};
template <>
struct Vec8<double> {
    __device__ static void load(const double *p, double (&v)[8])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double2 a = *reinterpret_cast<const double2 *>(p + 2 * i);
            v[2 * i] = a.x;
            v[2 * i + 1] = a.y;
        }
    }
    __device__ static void store(double *p, const double (&v)[8])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            *reinterpret_cast<double2 *>(p + 2 * i) = make_double2(v[2 * i], v[2 * i + 1]);
    }
};

// 8 consecutive samples starting at k0 (< cnt), zero past cnt. p is 16-byte aligned at k0.
template <typename T>
__device__ __forceinline__ void load8(const T *p, int k0, int cnt, T (&v)[8])
{
    if (k0 + 8 <= cnt) {
        Vec8<T>::load(p + k0, v);
    } else {
#pragma unroll
        for (int s = 0; s < 8; ++s)
            v[s] = (k0 + s < cnt) ? p[k0 + s] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void store8(T *p, int k0, int cnt, const T (&v)[8])
{
    if (k0 + 8 <= cnt) {
        Vec8<T>::store(p + k0, v);
    } else {
#pragma unroll
        for (int s = 0; s < 8; ++s)
            if (k0 + s < cnt)
                p[k0 + s] = v[s];
    }
}

// Step 1 on the tile in S.hs: extremum masks of this thread's 8 samples (maximum:
// h[k-1] < h[k] >= h[k+1]; minimum: h[k-1] > h[k] <= h[k+1]; never at the instance's
// end samples), their block-wide exclusive ranks, and the compacted knot positions
// env[e].kte[1 + rank]. Then, by all threads, the length, 1/length, slope and left value
// of every interval between two knots of the tile (cf[1..m-1]). Ends with the knot
// counts in S.cnt and a barrier.
template <typename R, int TILE, int NT>
__device__ __forceinline__ void find_knots(PassSmem<R, TILE, NT> &S, const R (&v)[8], int k0,
                                           int ts, int L, int cnt, uint32_t &MX, uint32_t &MN,
                                           int &bx, int &bn)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const R *hs = S.hs + 4;
    const R left = hs[k0 - 1], right = hs[k0 + 8];
    uint32_t up = 0, dn = 0; // bit s: h[k0+s] < h[k0+s+1] / h[k0+s] > h[k0+s+1]
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const R nx = s < 7 ? v[s + 1] : right;
        up |= (uint32_t)(v[s] < nx) << s;
        dn |= (uint32_t)(v[s] > nx) << s;
    }
    const uint32_t upl = (up << 1) | (uint32_t)(left < v[0]);
    const uint32_t dnl = (dn << 1) | (uint32_t)(left > v[0]);
    // valid samples: inside the tile's count and 1 <= global index <= L-2
    const int g0 = ts + k0;
    const int lo = max(0, 1 - g0), hi = min(min(8, cnt - k0), L - 1 - g0);
    const uint32_t valid = hi > lo ? (((1u << hi) - 1u) & ~((1u << lo) - 1u)) : 0u;
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
    if (lane == 31)
        S.wcnt[w] = incl;
    __syncthreads();
    uint32_t before = incl - packed, total = 0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {
        const uint32_t t = S.wcnt[ww];
        before += ww < w ? t : 0u;
        total += t;
    }
    bx = (int)(before & 0xffffu);
    bn = (int)(before >> 16);
    int ix = bx + 1, in = bn + 1;
    int *kx = S.env[0].kte, *kn = S.env[1].kte;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        if ((MX >> s) & 1u)
            kx[ix++] = k0 + s;
        if ((MN >> s) & 1u)
            kn[in++] = k0 + s;
    }
    const int m0 = (int)(total & 0xffffu), m1 = (int)(total >> 16);
    if (threadIdx.x == 0) {
        S.cnt[0] = m0;
        S.cnt[1] = m1;
    }
    __syncthreads();
    const int n0 = max(m0 - 1, 0), n1 = max(m1 - 1, 0);
    for (int idx = threadIdx.x; idx < n0 + n1; idx += NT) {
        const int e = idx < n0 ? 0 : 1;
        const int q = (idx < n0 ? idx : idx - n0) + 1;
        EnvSmem<R, TILE> &E = S.env[e];
        const int tl = E.kte[q], tr = E.kte[q + 1];
        const R yl = hs[tl];
        const R h = R(tr - tl), inv = rrcp(h);
        E.cf[q] = Coef<R>{(hs[tr] - yl) * inv, inv, h, yl};
    }
    __syncthreads();
}

// Step 2 for one envelope of the tile (one warp): natural-spline second derivatives M_j
// of the interior knots 1..m-2 given M_0 = MF and M_{m-1} = ML from the interface
// solve; row j: h_j M_{j-1} + 2 (h_j + h_{j+1}) M_j + h_{j+1} M_{j+1} = 6 (S_{j+1} - S_j),
// h_j and S_j the length and slope of interval j (precomputed in cf[j]). Writes the
// halved cubic of every interval q = 0..m to E.cf[q]. With EXPORT, instead eliminates
// the interior in terms of the unknown M_0 and M_{m-1} and returns M_1 (first) and
// M_{m-2} (last) as affine functions of them (m >= 3 required).
template <typename R, int TILE, bool EXPORT>
__device__ void envelope_solve(EnvSmem<R, TILE> &E, const R *hv, int m, const SolveVals<R> &sv,
                               R (&first)[3], R (&last)[3])
{
    const int lane = threadIdx.x & 31;
    const R MF = EXPORT ? R(0) : sv.MF, ML = EXPORT ? R(0) : sv.ML;
    const int n = m - 2; // interior unknowns; row i is knot i + 1
    if (!EXPORT && lane == 0) {
        // the intervals at the tile's ends: bracket knot -> knot 0, knot m-1 -> bracket
        auto T = [&](int j) { return E.kte[j + 1]; };
        auto Y = [&](int j) { return hv[E.kte[j + 1]]; };
        if (m == 0) {
            E.cf[0] = half_cubic<R>(T(-1), sv.yp, sv.Mp, T(0), sv.yn, sv.Mn);
        } else {
            E.cf[0] = half_cubic<R>(T(-1), sv.yp, sv.Mp, T(0), Y(0), MF);
            E.cf[m] = half_cubic<R>(T(m - 1), Y(m - 1), ML, T(m), sv.yn, sv.Mn);
            if (m == 2)
                E.cf[1] = half_cubic<R>(T(0), Y(0), MF, T(1), Y(1), ML);
        }
    }
    if (n <= 0)
        return;
    int Q = (n + 31) >> 5;
    Q |= 1;
    const int s = min(lane * Q, n), e = min(s + Q, n), q = e - s;
    SegElim<R> g;
    if (q >= 1) {
        // forward elimination of rows s..e-2 (knots s+1..e-1), the next interval's data
        // fetched one row ahead; the lane's last row (knot e) is kept for the reduction
        Coef<R> iv = E.cf[s + 1];
        R hA = iv.c2, SA = iv.c0;
        iv = E.cf[s + 2];
        R cprev = R(0), dprev = R(0), bprev = R(0);
        for (int j = s + 1; j < e; ++j) {
            const Coef<R> nxt = E.cf[j + 2];
            const R hB = iv.c2, SB = iv.c0;
            const R a = hA, c = hB, b = R(2) * (a + c), d = R(6) * (SB - SA);
            const bool f = j == s + 1;
            const R den = f ? b : b - a * cprev;
            const R inv = rrcp(den);
            cprev = c * inv;
            dprev = (f ? d : d - a * dprev) * inv;
            bprev = (f ? -a : -a * bprev) * inv;
            E.rw[j - 1] = Coef<R>{cprev, dprev, bprev, R(0)};
            hA = hB;
            SA = SB;
            iv = nxt;
        }
        g.al = hA;
        g.cl = iv.c2;
        g.bl = R(2) * (g.al + g.cl);
        g.dl = R(6) * (iv.c0 - SA);
        if (q >= 2) {
            g.alE = dprev;
            g.beE = bprev;
            g.gaE = -cprev;
            R xa = g.alE, xb = g.beE, xg = g.gaE;
            Coef<R> w = E.rw[max(e - 3, s)];
            for (int r = e - 3; r >= s; --r) {
                const Coef<R> wn = E.rw[max(r - 1, s)];
                xa = w.c1 - w.c0 * xa;
                xb = w.c2 - w.c0 * xb;
                xg = -w.c0 * xg;
                w = wn;
            }
            g.alS = xa;
            g.beS = xb;
            g.gaS = xg;
        }
    }
    const bool has_next = (q >= 1) && (e < n);
    if constexpr (EXPORT) {
        const R xl[3] = {R(0), R(1), R(0)}, xr[3] = {R(0), R(0), R(1)};
        R Z[3];
        warp_reduced_solve<R, 3>(g, q, has_next, xl, xr, Z);
        const int last_lane = (n - 1) / Q;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const R f = (k == 0 ? g.alS : R(0)) + g.beS * xl[k] + g.gaS * Z[k];
            first[k] = __shfl_sync(FULLMASK, f, 0);
            last[k] = __shfl_sync(FULLMASK, Z[k], last_lane);
        }
    } else {
        const R xl[1] = {MF}, xr[1] = {ML};
        R Z[1];
        warp_reduced_solve<R, 1>(g, q, has_next, xl, xr, Z);
        R Zp = __shfl_up_sync(FULLMASK, Z[0], 1);
        if (lane == 0)
            Zp = MF;
        if (q >= 1) {
            // back-substitution, descending, with the cubic of each interval as soon as
            // both of its second derivatives are known (interval j+1: knot j -> j+1)
            R xn = Z[0];
            if (e == n) {
                const Coef<R> st = E.cf[n + 1];
                E.cf[n + 1] = half_cubic_from(st.c3, xn, ML, st.c2, st.c1, st.c0);
            }
            Coef<R> w = E.rw[max(e - 2, 0)], st = E.cf[e];
            for (int j = e - 1; j >= s + 1; --j) {
                const Coef<R> wn = E.rw[max(j - 2, 0)], stn = E.cf[j];
                const R x = w.c1 + w.c2 * Zp - w.c0 * xn;
                E.cf[j + 1] = half_cubic_from(st.c3, x, xn, st.c2, st.c1, st.c0);
                xn = x;
                w = wn;
                st = stn;
            }
            const Coef<R> s1 = E.cf[s + 1];
            E.cf[s + 1] = half_cubic_from(s1.c3, Zp, xn, s1.c2, s1.c1, s1.c0);
        }
    }
}

// ---------------------------------------------------------------------------------
// One sifting pass over one tile. Grid: one CTA per tile of every running instance.
template <typename R, int TILE, int NT>
__global__ void __launch_bounds__(NT) k_pass(PassArgs pa)
{
    constexpr int NW = NT / 32;
    static_assert(TILE == 8 * NT && NW >= 2 && NW <= 32, "8 samples per thread, >= 2 warps");
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
    const int L = (int)in.L;
    const int lt = gt - in.tile0;
    const int ts = lt * TILE;
    const int cnt = min(TILE, L - ts);
    const bool hasL = ts > 0, hasR = ts + TILE < L;
    const R *hsrc = (const R *)in.h[hpar] + ts;
    R *hdst = (R *)in.h[hpar ^ 1] + ts;
    const double *rsrc = in.r[rpar] + ts;
    double *rdst = in.r[rpar ^ 1] + ts;
    const bool sift = mode == MODE_SIFT || mode == MODE_SIFT_COMMIT;
    const bool commit = mode == MODE_SIFT_COMMIT || mode == MODE_COMMIT;
    const int k0 = tid * 8;
    R *hs = S.hs + 4;

    R v[8], hn[8];
    R hcl = R(0), hcr = R(0); // current signal at the halo samples -1 and TILE
    if (mode != MODE_INIT) {
        load8(hsrc, k0, cnt, v);
        if (tid == 0 && hasL)
            hcl = hsrc[-1];
        if (tid == NT - 1 && hasR)
            hcr = hsrc[TILE];
    }

    R pn = R(0), pd = R(0);
    R hnl = hcl, hnr = hcr; // the new signal at the halo samples
    if (sift) {
        Vec8<R>::store(hs + k0, v);
        if (tid == 0)
            hs[-1] = hcl;
        if (tid == NT - 1)
            hs[TILE] = hcr;
        __syncthreads();
        uint32_t MX, MN;
        int bx, bn;
        find_knots<R, TILE, NT>(S, v, k0, ts, L, cnt, MX, MN, bx, bn);
        const TileSolve *so = in.tsol + 2 * lt;
        if (tid < 2) {
            EnvSmem<R, TILE> &E = S.env[tid];
            E.kte[0] = so[tid].tp - ts;
            E.kte[S.cnt[tid] + 1] = so[tid].tn - ts;
        }
        __syncthreads();
        if (warp < 2) {
            R f[3], l[3];
            envelope_solve<R, TILE, false>(S.env[warp], hs, S.cnt[warp],
                                           solve_vals(so[warp], R(0)), f, l);
        }
        __syncthreads();
        // Steps 2-4 at every sample: both envelopes (interval = knots at or before k),
        // their mean, the subtraction, and the SD partial sums
        const EnvSmem<R, TILE> &E0 = S.env[0], &E1 = S.env[1];
        int q0 = bx, q1 = bn;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            q0 += (MX >> s) & 1u;
            q1 += (MN >> s) & 1u;
            const int k = k0 + s;
            const R e0 = horner(E0.cf[q0], R(k - E0.kte[q0]));
            const R e1 = horner(E1.cf[q1], R(k - E1.kte[q1]));
            const R mean = radd(e0, e1);
            hn[s] = rsub(v[s], mean);
            if (k < cnt) {
                pn += mean * mean;
                pd += v[s] * v[s];
            }
        }
        // halo samples: interval 0 before the tile, interval m after it (where a knot on
        // the sample itself gives the knot value, as the neighbour computes it)
        if (tid == 0 && hasL) {
            const R mean = radd(horner(E0.cf[0], R(-1 - E0.kte[0])),
                                horner(E1.cf[0], R(-1 - E1.kte[0])));
            hnl = rsub(hcl, mean);
        }
        if (tid == NT - 1 && hasR) {
            const int m0 = S.cnt[0], m1 = S.cnt[1];
            const R e0 = E0.kte[m0 + 1] == TILE ? rmul(solve_vals(so[0], R(0)).yn, R(0.5))
                                                  : horner(E0.cf[m0], R(TILE - E0.kte[m0]));
            const R e1 = E1.kte[m1 + 1] == TILE ? rmul(solve_vals(so[1], R(0)).yn, R(0.5))
                                                  : horner(E1.cf[m1], R(TILE - E1.kte[m1]));
            hnr = rsub(hcr, radd(e0, e1));
        }
    } else {
#pragma unroll
        for (int s = 0; s < 8; ++s)
            hn[s] = v[s];
    }

    // Step 5 / Eq. (1): commit the IMF c, update the FP64 residue, restart from it
    if (commit || mode == MODE_INIT) {
        double r[8];
        load8(rsrc, k0, cnt, r);
        if (commit) {
            double rn[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                rn[s] = __dsub_rn(r[s], (double)hn[s]);
            }
            store8(rdst, k0, cnt, rn);
            R *imf = (R *)in.imf + (int64_t)imfc * in.imf_stride;
            if (in.imf_serialized) {
                store8(imf + ts, k0, cnt, hn);
            } else {
                const int64_t MD = in.M + in.D;
                const int p0 = ts + k0;
                int64_t i = p0 / MD, mm = p0 - i * MD;
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    if (k0 + s < cnt && mm < in.M)
                        imf[in.order == 0 ? i * in.M + mm : mm * in.N + i] = hn[s];
                    if (++mm == MD) {
                        mm = 0;
                        ++i;
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < 8; ++s)
                hn[s] = (R)rn[s];
        } else {
#pragma unroll
            for (int s = 0; s < 8; ++s)
                hn[s] = (R)r[s];
        }
        if (tid == 0 && hasL)
            hnl = (R)(commit ? __dsub_rn(rsrc[-1], (double)hnl) : rsrc[-1]);
        if (tid == NT - 1 && hasR)
            hnr = (R)(commit ? __dsub_rn(rsrc[TILE], (double)hnr) : rsrc[TILE]);
    }

    // Step 1 on the new signal and the per-tile elimination of its spline system
    if (sift)
        __syncthreads(); // the solve and the evaluation are done with hs and env
    Vec8<R>::store(hs + k0, hn);
    if (tid == 0)
        hs[-1] = hnl;
    if (tid == NT - 1)
        hs[TILE] = hnr;
    __syncthreads();
    {
        uint32_t MX, MN;
        int bx, bn;
        find_knots<R, TILE, NT>(S, hn, k0, ts, L, cnt, MX, MN, bx, bn);
    }
    if (warp < 2) {
        const int e = warp;
        const int m = S.cnt[e];
        const EnvSmem<R, TILE> &E = S.env[e];
        TileExport *rec = in.tex + 2 * lt + e;
        R f[3] = {R(0), R(0), R(0)}, l[3] = {R(0), R(0), R(0)};
        if (m >= 3)
            envelope_solve<R, TILE, true>(S.env[e], hs, m, SolveVals<R>{}, f, l);
        if (lane == 0) {
            rec->n = m;
            if (m >= 1) {
                const int ix[4] = {0, min(1, m - 1), max(m - 2, 0), m - 1};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = E.kte[ix[q] + 1];
                    rec->t[q] = ts + t;
                    put_slot(&rec->y[q], hs[t]);
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                put_slot(&rec->xa[q], f[q]);
                put_slot(&rec->xb[q], l[q]);
            }
        }
    }
    store8(hdst, k0, cnt, hn);
    if (tid == 0 && !hasL)
        in.taux[lt].h_first = (double)hn[0];
    if (!hasR && k0 <= cnt - 1 && cnt - 1 < k0 + 8) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
            if (k0 + s == cnt - 1)
                in.taux[lt].h_last = (double)hn[s];
    }
    if (sift) {
        pn = warp_sum(pn);
        pd = warp_sum(pd);
        if (lane == 0) {
            S.red[0][warp] = pn;
            S.red[1][warp] = pd;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                a += (double)S.red[0][w];
                b += (double)S.red[1][w];
            }
            in.taux[lt].sd_num = a;
            in.taux[lt].sd_den = b;
        }
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
// Per instance: stop test and state machine, then the reduced interface system of the
// spline solve for each envelope (warp 0: maxima, warp 1: minima), in FP64.
__global__ void __launch_bounds__(64) k_reduce(ReduceArgs ra)
{
    const int ii = ra.inst_list ? ra.inst_list[blockIdx.x] : (int)blockIdx.x;
    State *st = ra.state + ii;
    const int pm = st->mode;
    if (pm == MODE_DONE)
        return;
    const Inst &in = ra.inst[ii];
    const int e = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = in.ntiles;
    const int TQ = (nt + 31) / 32;
    const int ta = min(lane * TQ, nt), tb = min(ta + TQ, nt);
    const TileExport *tex = in.tex + e;
    int sn = 0, su = 0;
    for (int t = ta; t < tb; ++t) {
        const int n = tex[2 * t].n;
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
                a += in.taux[t].sd_num;
                b += in.taux[t].sd_den;
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
        const int64_t cap = in.rlen;
        Rn = in.rent + (int64_t)e * cap;
        double *dbl = in.rscr + (int64_t)e * 8 * cap;
        A = dbl;
        B = dbl + cap;
        C = dbl + 2 * cap;
        D = dbl + 3 * cap;
        Mv = dbl + 4 * cap;
        cpv = dbl + 5 * cap;
        dpv = dbl + 6 * cap;
        bpv = dbl + 7 * cap;
    }
    // tile-record values in the pass kernel's precision, widened to FP64
    const bool single = ra.single != 0;
    auto W = [single](const double &v) {
        return single ? (double)*reinterpret_cast<const float *>(&v) : v;
    };
    const int nl = ra.boundary == BND_MIRROR ? min(ra.mirror_knots, ntot) : 1;
    const int nr = nl;
    const int NR = nl + U + nr;
    {
        int p = nl + ubase;
        for (int t = ta; t < tb; ++t) {
            const TileExport &rc = tex[2 * t];
            if (rc.n == 1) {
                Rn[p++] = REntry{rc.t[0], t, RK_FL, 0, W(rc.y[0])};
            } else if (rc.n >= 2) {
                Rn[p++] = REntry{rc.t[0], t, RK_F, 0, W(rc.y[0])};
                Rn[p++] = REntry{rc.t[3], t, RK_L, 0, W(rc.y[3])};
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        const int64_t L = in.L;
        if (ra.boundary == BND_MIRROR) {
            // first two and last two knots of the whole signal, reflected about the ends
            const REntry k0 = Rn[nl];
            const TileExport &r0 = tex[2 * k0.tile];
            if (nl == 2) {
                int t1;
                double y1;
                if (r0.n >= 2) {
                    t1 = r0.t[1];
                    y1 = W(r0.y[1]);
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
            const TileExport &rl = tex[2 * kl.tile];
            const int Lm = (int)(2 * (L - 1));
            if (nr == 2) {
                int t2;
                double y2;
                if (rl.n >= 2) {
                    t2 = rl.t[2];
                    y2 = W(rl.y[2]);
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
            Rn[0] = REntry{0, -1, RK_FIXED, 0, in.taux[0].h_first};
            Rn[nl + U] = REntry{(int)(L - 1), -1, RK_FIXED, 0, in.taux[nt - 1].h_last};
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
                rc = &tex[2 * c.tile];
            const bool subR = c.kind == RK_F && rc->n >= 3;
            const bool subL = c.kind == RK_L && rc->n >= 3;
            if (subR) {
                tr = rc->t[1];
                yr = W(rc->y[1]);
            }
            if (subL) {
                tl = rc->t[2];
                yl = W(rc->y[2]);
            }
            const double hl = (double)c.t - tl, hr = tr - (double)c.t;
            const double a0 = hl, b0 = 2.0 * (hl + hr), c0 = hr;
            const double d0 = 6.0 * ((yr - c.y) * rrcp(hr) - (c.y - yl) * rrcp(hl));
            a = a0;
            b = b0;
            cc = c0;
            d = d0;
            if (subR) {
                b = b0 + c0 * W(rc->xa[1]);
                cc = c0 * W(rc->xa[2]);
                d = d0 - c0 * W(rc->xa[0]);
            }
            if (subL) {
                a = a0 * W(rc->xb[1]);
                b = b0 + a0 * W(rc->xb[2]);
                d = d0 - a0 * W(rc->xb[0]);
            }
        }
        A[p] = a;
        B[p] = b;
        C[p] = cc;
        D[p] = d;
    }
    __syncwarp();
    warp_tridiag<double>(NR, ScratchRows{A, B, C, D}, 0.0, 0.0, cpv, dpv, bpv,
                         [Mv](int i, double x) { Mv[i] = x; });
    __syncwarp();
    {
        int p = nl + ubase;
        for (int t = ta; t < tb; ++t) {
            const int n = tex[2 * t].n;
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
            so.f[0] = (float)so.MF;
            so.f[1] = (float)so.ML;
            so.f[2] = (float)so.yp;
            so.f[3] = (float)so.Mp;
            so.f[4] = (float)so.yn;
            so.f[5] = (float)so.Mn;
            so.pad[0] = so.pad[1] = 0;
            in.tsol[2 * t + e] = so;
            p += u;
        }
    }
}

} // namespace semd
