// Host runtime and C ABI of the GB300 Serial-EMD library: plans, workspaces, the
// pass loop, serialization (Sec. 3.2), de-serialization (Sec. 3.3) and the EEMD
// ensemble (Sec. 2.2). See semd_device.cuh for the sifting kernels.
#include "semd_runtime.h"
#include "semd_device.cuh"
#include "semd_reduce_cl.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

static_assert(sizeof(semd_params) == 80, "semd_params is part of the C ABI");

namespace semd {

static thread_local std::string g_plan_create_error;

// ----------------------------------------------------------------- helper kernels

// Sec. 3.2 serialization, one CTA per tile: x[i(M+D)+m] = X(i, m) for m < M and, for
// the D transition samples between signal i and i+1 (0-based r),
// x = (r+1)/(D+1) * X(i+1, D-1-r) + (D-r)/(D+1) * X(i, M-1-r). Written in FP64 to r0.
// Only instances that have not started (state MODE_INIT) are serialized.
template <typename R>
__device__ __forceinline__ double serial_sample(const R *X, int64_t M, int64_t N, int64_t D,
                                                int order, int64_t p)
{
    // serialized lengths are below 2^30 (plan validation): 32-bit division
    const uint32_t md = (uint32_t)(M + D);
    const int64_t i = (uint32_t)p / md, m = p - i * (int64_t)md;
    if (m < M)
        return (double)X[order == 0 ? i * M + m : m * N + i];
    const int64_t r = m - M;
    const int64_t ma = D - 1 - r, mb = M - 1 - r;
    const double xa = (double)X[order == 0 ? (i + 1) * M + ma : ma * N + (i + 1)];
    const double xb = (double)X[order == 0 ? i * M + mb : mb * N + i];
    const double a = (double)(r + 1) / (double)(D + 1);
    const double af = (double)(D - r) / (double)(D + 1);
    return __dadd_rn(__dmul_rn(xa, a), __dmul_rn(xb, af));
}

template <typename R>
__global__ void k_serialize(const Inst *inst, const State *state, const int32_t *tile_inst,
                            int tile, int only_first)
{
    const int gt = blockIdx.x, ii = tile_inst[gt];
    if ((only_first && ii != 0) || state[ii].mode != MODE_INIT)
        return;
    const Inst &in = inst[ii];
    const int64_t ts = (int64_t)(gt - in.tile0) * tile;
    const int64_t cnt = min((int64_t)tile, in.L - ts);
    const R *X = (const R *)in.x;
    for (int64_t idx = threadIdx.x; idx < cnt; idx += blockDim.x)
        in.r[0][ts + idx] = serial_sample<R>(X, in.M, in.N, in.D, in.order, ts + idx);
}

// EEMD beta = rel * population std of the serialized x (Sec. 2.2 Step 1): the mean, then
// the mean squared deviation from it, each a sum over kStdBlocks CTAs in a fixed order
// (results do not depend on timing). part holds 2 kStdBlocks partial sums.
constexpr int kStdBlocks = 256;
constexpr int kStdThreads = 256;

// Sum of the CTA's threads' values in a fixed tree order (every thread gets the total).
__device__ double block_sum_fixed(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double t = sh[0];
    __syncthreads();
    return t;
}

// Stage 0: CTA b's share of sum x. Stage 1: the mean from the stage-0 partials, CTA b's
// share of sum (x - mean)^2. Stage 2 (one CTA): beta from the stage-1 partials.
__global__ void __launch_bounds__(kStdThreads) k_std(const Inst *inst, double rel, double *beta,
                                                     double *part, int stage)
{
    __shared__ double sh[kStdThreads];
    const double *x = inst[0].r[0];
    const int64_t L = inst[0].L;
    const int64_t stride = (int64_t)kStdBlocks * kStdThreads;
    if (stage == 2) {
        double v = 0.0;
        for (int i = threadIdx.x; i < kStdBlocks; i += blockDim.x)
            v += part[kStdBlocks + i];
        const double t = block_sum_fixed(v, sh);
        if (threadIdx.x == 0)
            *beta = rel * sqrt(t / (double)L);
        return;
    }
    double mean = 0.0;
    if (stage == 1) {
        double v = 0.0;
        for (int i = threadIdx.x; i < kStdBlocks; i += blockDim.x)
            v += part[i];
        mean = block_sum_fixed(v, sh) / (double)L;
    }
    double s = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)kStdThreads + threadIdx.x; k < L; k += stride) {
        const double d = stage == 1 ? x[k] - mean : x[k];
        s += stage == 1 ? d * d : d;
    }
    const double t = block_sum_fixed(s, sh);
    if (threadIdx.x == 0)
        part[stage * kStdBlocks + blockIdx.x] = t;
}

// One Philox4x32-10 block (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds of two 32 x 32 -> 64-bit products of counter
// words with the round multipliers, the high halves mixed with the other counter words and
// the round key, the key bumped by a Weyl sequence between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// White noise drawn by the library (Sec. 2.2 asks for white noise of a given deviation):
// realization m, serialized sample p takes word p mod 4 of the Philox block with counter
// (p div 4, m, 0, 0) and key (seed low word, seed high word); the word u gives the odd
// integer i = 2 (u >> 9) - (2^23 - 1) and the sample i * sqrt(3) / 2^23, uniform on
// (-sqrt 3, sqrt 3) with zero mean and unit variance.
__device__ __forceinline__ double white_value(uint32_t u)
{
    const int32_t i = (int32_t)(2u * (u >> 9)) - 8388607;
    return __dmul_rn((double)i, 1.7320508075688772 / 8388608.0);
}
__device__ __forceinline__ double white_sample(uint64_t seed, int m, int64_t p)
{
    const uint4 b = philox4x32_10(make_uint4((uint32_t)(p >> 2), (uint32_t)m, 0u, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const int j = (int)(p & 3);
    return white_value(j == 0 ? b.x : j == 1 ? b.y : j == 2 ? b.z : b.w);
}

// x^(m) = x + beta w^(m) for the trials m0 + blockIdx.y (Sec. 2.2 Step 1); trial 0 holds
// x on entry, so the host runs trials 1.. first and trial 0 (in place) last. The noise is
// the caller's (inst[0].noise) or, when that is null, drawn here from the seed: a warp
// owns 128 consecutive samples of one trial, lane l computes the Philox block of samples
// 128 g + 4 l .. + 3, and the words are passed by shuffles so that in round j lane l writes
// sample 128 g + 32 j + l (coalesced).
template <typename R>
__global__ void k_add_noise(const Inst *inst, int m0, const double *beta, uint64_t seed)
{
    const int64_t L = inst[0].L;
    const R *w = (const R *)inst[0].noise;
    const double b = *beta;
    const int m = m0 + (int)blockIdx.y;
    const int lane = threadIdx.x & 31;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int64_t nw = (L + 127) >> 7;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double *x0 = inst[0].r[0];
    double *dst = inst[m].r[0];
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nw; g += stride) {
        const int64_t p0 = (g << 7) + lane;
        double x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            x[j] = p0 + 32 * j < L ? x0[p0 + 32 * j] : 0.0;
        if (w) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t p = p0 + 32 * j;
                if (p < L)
                    dst[p] = __dadd_rn(x[j], __dmul_rn(b, (double)w[(int64_t)m * L + p]));
            }
            continue;
        }
        const uint4 blk =
            philox4x32_10(make_uint4((uint32_t)((g << 5) + lane), (uint32_t)m, 0u, 0u), key);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            // sample 128 g + 32 j + lane: block 32 g + 8 j + lane / 4, word lane mod 4
            const int src = 8 * j + (lane >> 2);
            const uint32_t u0 = __shfl_sync(FULLMASK, blk.x, src);
            const uint32_t u1 = __shfl_sync(FULLMASK, blk.y, src);
            const uint32_t u2 = __shfl_sync(FULLMASK, blk.z, src);
            const uint32_t u3 = __shfl_sync(FULLMASK, blk.w, src);
            const int q = lane & 3;
            const uint32_t u = q == 0 ? u0 : q == 1 ? u1 : q == 2 ? u2 : u3;
            const int64_t p = p0 + 32 * j;
            if (p < L)
                dst[p] = __dadd_rn(x[j], __dmul_rn(b, white_value(u)));
        }
    }
}

// Grid of k_add_noise for a signal of ntiles tiles and `trials` trials: a warp per 128
// samples (8 per CTA) in x, a trial per y.
static dim3 noise_grid(int64_t ntiles, int tile, int trials)
{
    const int64_t warps = (ntiles * tile + 127) / 128;
    return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 1 << 16)),
                (unsigned)trials);
}

// Sec. 3.3 for the residue, and zero-fill of the IMF slots past the produced count, for
// instances whose decomposition has ended (state MODE_DONE).
template <typename R>
__global__ void k_finalize(const Inst *inst, const State *state, const int32_t *tile_inst,
                           int tile, int K)
{
    const int gt = blockIdx.x, ii = tile_inst[gt];
    const Inst &in = inst[ii];
    if (in.imf_serialized || state[ii].mode != MODE_DONE)
        return;
    const int n = state[ii].imf_count;
    const double *r = in.r[state[ii].rpar];
    const int64_t ts = (int64_t)(gt - in.tile0) * tile;
    const int64_t cnt = min((int64_t)tile, in.L - ts);
    R *imf = (R *)in.imf;
    for (int64_t idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
        const int64_t p = ts + idx;
        int64_t dst;
        if (!deser_index(p, in.M, in.N, in.D, in.order, dst))
            continue;
        if (in.res)
            in.res[dst] = r[p];
        for (int k = n; k < K; ++k)
            imf[(int64_t)k * in.imf_stride + dst] = R(0);
    }
}

// EEMD Step 3: average the trials' IMFs (zeros where a trial has fewer) and residues, in
// trial order, then de-serialize (Sec. 3.3). FP64 plans sum in FP64. FP32 plans sum the
// single-precision IMF values in float-float arithmetic (an unevaluated pair of floats,
// about 48 significant bits: as accurate as the FP64 sum for these inputs, without the
// narrow FP64 pipe); the residues are FP64 in both. A thread takes 4 consecutive samples
// (16- or 32-byte loads of each trial's IMF row) of one IMF k = blockIdx.y (k = K: the
// residue), a CTA 1024 samples; the trials' IMF counts and residue arrays are read once per
// CTA into shared memory (the first kAvgShared trials).
constexpr int kAvgShared = 512;
constexpr int kAvgPer = 4;
template <typename R>
__global__ void k_eemd_average(const Inst *inst, const State *state, int trials, int K,
                               const R *scratch)
{
    __shared__ int ncnt[kAvgShared];
    __shared__ const double *rptr[kAvgShared];
    for (int m = threadIdx.x; m < min(trials, kAvgShared); m += blockDim.x) {
        ncnt[m] = state[m].imf_count;
        rptr[m] = inst[m].r[state[m].rpar];
    }
    __syncthreads();
    const Inst &in = inst[0];
    const int k = blockIdx.y;
    const int64_t L = in.L;
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kAvgPer;
    if (p0 >= L)
        return;
    const int n = (int)min((int64_t)kAvgPer, L - p0); // the tail thread may have fewer
    int64_t dst[kAvgPer];
    bool keep[kAvgPer];
#pragma unroll
    for (int j = 0; j < kAvgPer; ++j)
        keep[j] = j < n && deser_index(p0 + j, in.M, in.N, in.D, in.order, dst[j]);
    if (k == K) { // the residues
        double *res = in.avg_res;
        if (!res)
            return;
        double acc[kAvgPer] = {};
#pragma unroll 4
        for (int m = 0; m < trials; ++m) {
            const double *r = (m < kAvgShared ? rptr[m] : inst[m].r[state[m].rpar]) + p0;
#pragma unroll
            for (int j = 0; j < kAvgPer; ++j)
                acc[j] += j < n ? r[j] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kAvgPer; ++j)
            if (keep[j])
                res[dst[j]] = acc[j] / (double)trials;
        return;
    }
    auto count_of = [&](int m) { return m < kAvgShared ? ncnt[m] : state[m].imf_count; };
    R *out = (R *)in.avg_imf + (int64_t)k * in.M * in.N;
    const int64_t step = (int64_t)K * in.imf_stride; // one trial's IMF block
    const R *src = scratch + (int64_t)k * in.imf_stride + p0;
    double sum[kAvgPer];
    if constexpr (sizeof(R) == 4) {
        FFSum acc[kAvgPer];
#pragma unroll 4
        for (int m = 0; m < trials; ++m) {
            float v[kAvgPer];
            if (n == kAvgPer) {
                vload<kAvgPer>(src + m * step, v);
            } else {
#pragma unroll
                for (int j = 0; j < kAvgPer; ++j)
                    v[j] = j < n ? src[m * step + j] : 0.f;
            }
            if (k < count_of(m)) {
#pragma unroll
                for (int j = 0; j < kAvgPer; ++j)
                    acc[j].add(v[j], 0.f);
            }
        }
#pragma unroll
        for (int j = 0; j < kAvgPer; ++j)
            sum[j] = (double)acc[j].hi + (double)acc[j].lo;
    } else {
        double acc[kAvgPer] = {};
#pragma unroll 4
        for (int m = 0; m < trials; ++m) {
            double v[kAvgPer];
            if (n == kAvgPer) {
                vload<kAvgPer>(src + m * step, v);
            } else {
#pragma unroll
                for (int j = 0; j < kAvgPer; ++j)
                    v[j] = j < n ? src[m * step + j] : 0.0;
            }
            if (k < count_of(m)) {
#pragma unroll
                for (int j = 0; j < kAvgPer; ++j)
                    acc[j] += v[j];
            }
        }
#pragma unroll
        for (int j = 0; j < kAvgPer; ++j)
            sum[j] = acc[j];
    }
#pragma unroll
    for (int j = 0; j < kAvgPer; ++j)
        if (keep[j])
            out[dst[j]] = (R)(sum[j] / (double)trials);
}

// One EEMD realization's IMFs and residue as the last decomposition left them (Sec. 2.2:
// trial m is the EMD of x + beta w^(m)), de-serialized (Sec. 3.3); IMF slots past the
// trial's count are zero.
template <typename R>
__global__ void k_eemd_trial(const Inst *inst, const State *state, int m, int K, const R *scratch,
                             R *out, double *res)
{
    const Inst &in = inst[m];
    const int n = state[m].imf_count;
    const double *r = in.r[state[m].rpar];
    const int64_t MN = in.M * in.N;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < in.L;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t dst;
        if (!deser_index(p, in.M, in.N, in.D, in.order, dst))
            continue;
        for (int k = 0; k < K; ++k)
            out[(int64_t)k * MN + dst] =
                k < n ? scratch[((int64_t)m * K + k) * in.imf_stride + p] : R(0);
        if (res)
            res[dst] = r[p];
    }
}

// ------------------------------------------------------------- CEEMDAN (Sec. 2.2)
//
// Stage k (k = 0 .. K-1) of a CEEMDAN call: the IMF-start test and beta_k on r_k, the
// trials' inputs r_k + beta_k E_k(w^(m)) (E_0(w) = w), the first EMD mode of every trial
// (the sifting kernels with one IMF), then mode k+1 = the trial average and
// r_{k+1} = r_k - mode.

// After the EMD of the noise realizations: keep each realization's mode count (its modes
// past the count are zero) and point every trial's IMF output at the scratch slot K-1,
// which no stage reads (stage k reads slot k-1 <= K-2), for the stages' first modes.
__global__ void k_ce_setup(const CeArgs *ca, Inst *inst, const State *state, CeState *cs,
                           int noise_ran, int elem)
{
    const CeArgs &a = *ca;
    for (int m = threadIdx.x; m < a.trials; m += blockDim.x) {
        a.ncount[m] = noise_ran ? state[m].imf_count : 0;
        inst[m].imf = (char *)a.E + (size_t)((int64_t)m * a.K + (a.K - 1)) * a.slot * elem;
    }
    if (threadIdx.x == 0) {
        cs->beta = 0.0;
        cs->done = 0;
        cs->n = 0;
        cs->mean = 0.0;
        cs->arrived[0] = cs->arrived[1] = 0;
    }
}

// r_0 = the serialized input (Sec. 3.2).
template <typename R>
__global__ void k_ce_serialize(const CeArgs *ca)
{
    const CeArgs &a = *ca;
    const R *X = (const R *)a.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.L;
         p += (int64_t)gridDim.x * blockDim.x)
        a.r[p] = serial_sample<R>(X, a.M, a.N, a.D, a.order, p);
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULLMASK, v, o);
    __syncthreads(); // sh may still be read by a previous call
    if (lane == 0)
        sh[warp] = v;
    __syncthreads();
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}

// Stage test of r_k in two passes over blocks of kCeTestSpan samples, each ending in the
// last block to finish (a counter, no waiting): pass 0 sums r_k and the last block forms
// the mean; pass 1 sums (r_k - mean)^2 and counts extrema (the rule of Sec. 2.1 Step 1),
// and its last block takes the IMF-start test (n_max >= 1, n_min >= 1, n_max + n_min >= 3;
// when it fails this and every later stage is empty) and beta_k = rel * population std of
// r_k. The partials are combined in block order, so the result does not depend on timing.
__global__ void __launch_bounds__(256) k_ce_stage_test(const CeArgs *ca, CeState *cs,
                                                       CePart *part, int pass)
{
    if (cs->done)
        return;
    const CeArgs &a = *ca;
    const double *r = a.r;
    const int64_t L = a.L;
    const int64_t b0 = (int64_t)blockIdx.x * kCeTestSpan;
    const int64_t b1 = min(b0 + (int64_t)kCeTestSpan, L);
    __shared__ double shd[32];
    __shared__ int shi[32];
    __shared__ bool last;
    const double mean = pass == 0 ? 0.0 : cs->mean;
    double s = 0.0;
    int nmax = 0, nmin = 0;
    for (int64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
        const double c = r[k];
        if (pass == 0) {
            s += c;
        } else {
            s += (c - mean) * (c - mean);
            if (k >= 1 && k + 1 < L) {
                const double l = r[k - 1], rr = r[k + 1];
                nmax += (l < c && c >= rr) ? 1 : 0;
                nmin += (l > c && c <= rr) ? 1 : 0;
            }
        }
    }
    s = block_sum(s, shd);
    if (pass == 1) {
        nmax = block_sum(nmax, shi);
        nmin = block_sum(nmin, shi);
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = CePart{s, nmax, nmin};
        __threadfence();
        last = atomicAdd(&cs->arrived[pass], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int64_t xa = 0, xb = 0;
        for (unsigned q = 0; q < gridDim.x; ++q) { // L2 reads: other blocks wrote them
            t += __ldcg(&part[q].s);
            xa += __ldcg(&part[q].nmax);
            xb += __ldcg(&part[q].nmin);
        }
        cs->arrived[pass] = 0;
        if (pass == 0) {
            cs->mean = t / (double)L;
        } else if (xa >= 1 && xb >= 1 && xa + xb >= 3) {
            cs->n += 1;
            cs->beta = a.rel * sqrt(t / (double)L);
        } else {
            cs->done = 1;
        }
    }
}

// The trials' stage inputs r_k + beta_k E_k(w^(m)) as their residues for the INIT pass,
// one trial per grid row; for an empty stage every trial is marked done instead (its
// first mode counts as zero).
template <typename R>
__global__ void k_ce_stage_init(const CeArgs *ca, const Inst *inst, State *state,
                                const CeState *cs, int stage)
{
    const CeArgs &a = *ca;
    const int m = blockIdx.y;
    if (cs->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            state[m].mode = MODE_DONE;
        return;
    }
    const double beta = cs->beta;
    const R *e = stage == 0 ? (const R *)a.noise + (int64_t)m * a.L
                 : stage - 1 < a.ncount[m]
                     ? (const R *)a.E + ((int64_t)m * a.K + (stage - 1)) * a.slot
                     : nullptr;
    double *dst = inst[m].r[0];
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.L;
         p += (int64_t)gridDim.x * blockDim.x)
        dst[p] = __dadd_rn(a.r[p], __dmul_rn(beta, e ? (double)e[p] : 0.0));
}

// Mode k+1 = the average of the trials' first modes (zero for a trial without one), in
// FP64; r_{k+1} = r_k - mode (Step 3); the mode de-serialized (Sec. 3.3). A block covers
// 32 samples with 8 warps: warp g sums the trials m = g, g + 8, ... in order, then the 8
// partial sums are added in warp order (a fixed order, independent of timing).
constexpr int kCeAvgGroups = 8;
template <typename R>
__global__ void __launch_bounds__(32 * kCeAvgGroups)
    k_ce_average(const CeArgs *ca, const Inst *inst, const State *state, int stage)
{
    const CeArgs &a = *ca;
    __shared__ double part[kCeAvgGroups][32];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (p < a.L)
        for (int m = g; m < a.trials; m += kCeAvgGroups)
            if (state[m].imf_count >= 1)
                acc += (double)((const R *)inst[m].imf)[p];
    part[g][lane] = acc;
    __syncthreads();
    if (g != 0 || p >= a.L)
        return;
#pragma unroll
    for (int q = 1; q < kCeAvgGroups; ++q)
        acc += part[q][lane];
    const double c = acc / (double)a.trials;
    a.r[p] = a.r[p] - c;
    int64_t dst;
    if (deser_index(p, a.M, a.N, a.D, a.order, dst))
        ((R *)a.modes)[(int64_t)stage * a.M * a.N + dst] = (R)c;
}

// The final residue, de-serialized (Sec. 3.3).
__global__ void k_ce_finish(const CeArgs *ca)
{
    const CeArgs &a = *ca;
    if (!a.res)
        return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.L;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t dst;
        if (deser_index(p, a.M, a.N, a.D, a.order, dst))
            a.res[dst] = a.r[p];
    }
}

// Standalone extrema (Sec. 2.1 Step 1): per-tile counts, then ordered writes.
template <typename R>
__global__ void k_extrema_tiles(const R *h, int64_t L, int tile, const int32_t *base,
                                int32_t *counts, int32_t *tmax, int32_t *tmin)
{
    const int64_t ts = (int64_t)blockIdx.x * tile;
    const int64_t cnt = min((int64_t)tile, L - ts);
    if (threadIdx.x != 0)
        return;
    int a = 0, b = 0;
    int oa = base ? base[2 * blockIdx.x] : 0, ob = base ? base[2 * blockIdx.x + 1] : 0;
    for (int64_t k = ts; k < ts + cnt; ++k) {
        if (k < 1 || k > L - 2)
            continue;
        const R l = h[k - 1], c = h[k], r = h[k + 1];
        if (l < c && c >= r) {
            if (base)
                tmax[oa + a] = (int32_t)k;
            ++a;
        }
        if (l > c && c <= r) {
            if (base)
                tmin[ob + b] = (int32_t)k;
            ++b;
        }
    }
    if (!base) {
        counts[2 * blockIdx.x] = a;
        counts[2 * blockIdx.x + 1] = b;
    }
}

template <typename R>
__global__ void k_to_double(const R *h, int64_t L, double *r)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < L;
         p += (int64_t)gridDim.x * blockDim.x)
        r[p] = (double)h[p];
}

// ------------------------------------------------------------------ plan helpers

// The pass kernel for each supported tile: 128 / 256 / 512 samples per warp (4, 8, 16 per
// lane), kPassWarps warps per CTA, in two variants. Variant 0 (throughput) stages each
// warp's next tile in shared memory while the current one computes; for FP32 with
// 256-sample tiles it is compiled for four resident CTAs per SM (a few spilled bytes).
// Variant 1 (latency: launches with about one tile per warp) only prefetches into L2, a
// smaller kernel; FP32 256-sample tiles compile it for three CTAs per SM (no spills).
template <typename R, int TILE, int VAR>
static constexpr int pass_minb() { return (sizeof(R) == 4 && TILE == 256) ? (VAR == 0 ? 4 : 3) : 1; }
template <typename R, int TILE, int VAR>
static constexpr auto pass_kernel()
{
    return k_pass<R, TILE / 32, kPassWarps, pass_minb<R, TILE, VAR>(), VAR == 0>;
}

template <typename R, int TILE, int VAR>
static constexpr size_t pass_smem()
{
    return kPassWarps * (sizeof(WarpPool<R, TILE>) + (VAR == 0 ? sizeof(StageBuf<R, TILE>) : 0));
}

template <typename R, int TILE, int VAR>
static cudaError_t pass_attr_one()
{
    return cudaFuncSetAttribute(pass_kernel<R, TILE, VAR>(),
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pass_smem<R, TILE, VAR>());
}

// Which cluster shapes of the interface solve the current device can hold: per precision,
// device, cluster size (2, 4, 8, 16) and shared memory (up to 116 KB per CTA, or up to the
// opt-in maximum): 1 yes, 2 no. Filled once per precision and device, under a lock, when
// the kernel attributes are set (plan and server creation), so that no query runs while a
// stream is being captured; the ready flag is published after every entry.
constexpr int kClDevMax = 64;
static std::atomic<int> g_cluster_fit[2][kClDevMax][4][2];
static std::atomic<int> g_cluster_fit_ready[2][kClDevMax];
static std::mutex g_cluster_fit_mu;

template <typename R>
static void query_cluster_fit(int dev)
{
    for (int lc = 0; lc < 4; ++lc) {
        for (int big = 0; big < 2; ++big) {
            const unsigned CL = 2u << lc;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(CL);
            cfg.blockDim = dim3(kRedThreads);
            cfg.dynamicSmemBytes = big ? kClSmemOptin - 1024 : 116 * 1024;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = CL;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int n = 0;
            const bool ok =
                cudaOccupancyMaxActiveClusters(&n, k_reduce_cl<R>, &cfg) == cudaSuccess && n > 0;
            cudaGetLastError(); // a refused query leaves no error behind
            g_cluster_fit[sizeof(R) == 8][dev][lc][big].store(ok ? 1 : 2,
                                                               std::memory_order_relaxed);
        }
    }
}

// Whether a cluster of CL CTAs with `smem` bytes of shared memory each fits on the device.
template <typename R>
static bool cluster_fits(int CL, size_t smem)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kClDevMax)
        return false;
    if (!g_cluster_fit_ready[sizeof(R) == 8][dev].load(std::memory_order_acquire))
        return false;
    const int lc = CL == 2 ? 0 : CL == 4 ? 1 : CL == 8 ? 2 : 3;
    return g_cluster_fit[sizeof(R) == 8][dev][lc][smem > 116 * 1024 ? 1 : 0].load(
               std::memory_order_relaxed) == 1;
}

template <typename R>
static cudaError_t set_smem_attr()
{
    cudaError_t e = pass_attr_one<R, 128, 0>();
    if (e == cudaSuccess)
        e = pass_attr_one<R, 128, 1>();
    if (e == cudaSuccess)
        e = pass_attr_one<R, 256, 0>();
    if (e == cudaSuccess)
        e = pass_attr_one<R, 256, 1>();
    if (e == cudaSuccess)
        e = pass_attr_one<R, 512, 0>();
    if (e == cudaSuccess)
        e = pass_attr_one<R, 512, 1>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_reduce<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kReduceSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_reduce<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)reduce_smem_bytes(kRedSmallRows, sizeof(R)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_reduce<R, true, kRedThreadsTiny>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)reduce_smem_bytes(reduce_len(kRedThreadsTiny), sizeof(R)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_reduce_cl<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kClSmemOptin - 1024));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_reduce_cl<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int dev = 0;
    if (e == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kClDevMax &&
        !g_cluster_fit_ready[sizeof(R) == 8][dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lk(g_cluster_fit_mu);
        if (!g_cluster_fit_ready[sizeof(R) == 8][dev].load(std::memory_order_relaxed)) {
            query_cluster_fit<R>(dev);
            g_cluster_fit_ready[sizeof(R) == 8][dev].store(1, std::memory_order_release);
        }
    }
    return e;
}

// CTAs of a pass kernel that fit on one SM of the current device at once, and the
// device's SM count, computed once per device.
template <typename R, int TILE, int VAR>
static void pass_residency(int &per_sm, int &sms)
{
    constexpr int kMaxDev = 64;
    // [1] (SMs) is stored before [0] (CTAs per SM), which a reader checks first
    static std::atomic<int> cache[kMaxDev][2];
    int dev = 0;
    per_sm = 1;
    sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
        return;
    int ps = cache[dev][0].load(std::memory_order_acquire);
    if (ps == 0) {
        int a = 0, b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, pass_kernel<R, TILE, VAR>(),
                                                          32 * kPassWarps,
                                                          pass_smem<R, TILE, VAR>()) != cudaSuccess ||
            cudaDeviceGetAttribute(&b, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return;
        cache[dev][1].store(std::max(b, 1), std::memory_order_relaxed);
        cache[dev][0].store(std::max(a, 1), std::memory_order_release);
        ps = std::max(a, 1);
    }
    per_sm = ps;
    sms = cache[dev][1].load(std::memory_order_relaxed);
}

template <typename R>
static void pass_residency_of(int tile, int variant, int &per_sm, int &sms)
{
    if (tile == 128)
        variant == 1 ? pass_residency<R, 128, 1>(per_sm, sms) : pass_residency<R, 128, 0>(per_sm, sms);
    else if (tile == 512)
        variant == 1 ? pass_residency<R, 512, 1>(per_sm, sms) : pass_residency<R, 512, 0>(per_sm, sms);
    else
        variant == 1 ? pass_residency<R, 256, 1>(per_sm, sms) : pass_residency<R, 256, 0>(per_sm, sms);
}

int pass_ctas_per_sm_max(size_t elem, int tile, int variant)
{
    int per_sm = 1, sms = 152;
    if (elem == 8)
        pass_residency_of<double>(tile, variant, per_sm, sms);
    else
        pass_residency_of<float>(tile, variant, per_sm, sms);
    return per_sm;
}

// Launches with programmatic stream serialization: the kernel's CTAs may start while the
// previous kernel of the stream finishes (each waits in pdl_wait before reading its
// results), which hides the launch gap between the passes and the interface solves.
// Set while the body of a device-decided sifting loop is captured: kernels inside a
// conditional graph node are launched without programmatic stream serialization.
static thread_local bool g_plain_launches = false;

template <typename K, typename A>
static void launch_pdl(K kernel, unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       const A &arg)
{
    if (g_plain_launches) {
        kernel<<<grid, block, smem, s>>>(arg);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, arg);
}

// The persistent pass grid: at most ctas_per_sm CTAs per SM (0 or more than fit: as many
// as fit), and never more CTAs than the launch has tiles for.
template <typename R, int TILE, int VAR>
static void launch_pass_t(PassArgs pa, int64_t ntiles, int ctas_per_sm, cudaStream_t s)
{
    pa.ntiles = ntiles;
    int per_sm, sms;
    pass_residency<R, TILE, VAR>(per_sm, sms);
    if (ctas_per_sm > 0)
        per_sm = std::min(per_sm, ctas_per_sm);
    const int64_t grid =
        std::min((ntiles + kPassWarps - 1) / kPassWarps, (int64_t)per_sm * sms);
    launch_pdl(pass_kernel<R, TILE, VAR>(), (unsigned)grid, 32 * kPassWarps,
               pass_smem<R, TILE, VAR>(), s, pa);
}

template <typename R>
static void launch_pass_tiles(int tile, int variant, int ctas_per_sm, const PassArgs &pa,
                              int64_t ntiles, cudaStream_t s)
{
    if (tile == 128)
        variant == 1 ? launch_pass_t<R, 128, 1>(pa, ntiles, ctas_per_sm, s)
                     : launch_pass_t<R, 128, 0>(pa, ntiles, ctas_per_sm, s);
    else if (tile == 512)
        variant == 1 ? launch_pass_t<R, 512, 1>(pa, ntiles, ctas_per_sm, s)
                     : launch_pass_t<R, 512, 0>(pa, ntiles, ctas_per_sm, s);
    else
        variant == 1 ? launch_pass_t<R, 256, 1>(pa, ntiles, ctas_per_sm, s)
                     : launch_pass_t<R, 256, 0>(pa, ntiles, ctas_per_sm, s);
}

static size_t reduce_smem(const ReduceArgs &ra)
{
    return ra.smem_entries > 0 ? reduce_smem_bytes(ra.smem_entries, ra.single ? 4 : 8) : 0;
}

// SM count of the current device, looked up once per device.
static int device_sms()
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
        return 152;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 152;
        n = std::max(n, 1);
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// One CTA per instance and envelope. When the shared scratch holds every instance's
// system (smem_entries, sized for the launch's longest instance, bounds each system's
// rows) and that is at most kRedSmallRows rows, the small-system kernel runs. When the
// longest instance has at most kRedThreadsTiny tiles and the launch has more CTAs than the
// 256-thread small form keeps resident at once (its register budget: 3 per SM in FP32, 2
// in FP64), its 64-thread form runs instead (one thread per tile, four times the resident
// CTAs); a launch that fits in one wave keeps the 256-thread form, whose phases over the
// rows of a system have more threads.
// The cluster kernel: ra.cl CTAs per instance and envelope, one cluster each, launched
// with programmatic dependent launch like the other kernels of the sifting loop (its CTAs
// take the SMs the pass kernel leaves, and wait for it to finish before reading).
template <typename R>
static void launch_reduce_cl(const ReduceArgs &ra, int ninst, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * ninst * ra.cl));
    cfg.blockDim = dim3(kRedThreads);
    cfg.dynamicSmemBytes = cl_smem_bytes<R>(ra.cl_entries);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ra.cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_plain_launches ? 1 : 2;
    cudaLaunchKernelEx(&cfg, k_reduce_cl<R>, ra);
}

template <typename R>
static void launch_reduce(const ReduceArgs &ra, int ninst, cudaStream_t s)
{
    if (ra.run_cl)
        launch_reduce_cl<R>(ra, ninst, s);
    if (!ra.run_single)
        return;
    const int64_t wave = (int64_t)(sizeof(R) == 4 ? 3 : 2) * device_sms();
    if (ra.smem_entries > 0 && ra.smem_entries <= reduce_len(kRedThreadsTiny) && 2 * ninst > wave)
        launch_pdl(k_reduce<R, true, kRedThreadsTiny>, (unsigned)(2 * ninst), kRedThreadsTiny,
                   reduce_smem(ra), s, ra);
    else if (ra.smem_entries > 0 && ra.smem_entries <= kRedSmallRows)
        launch_pdl(k_reduce<R, true>, (unsigned)(2 * ninst), kRedThreads, reduce_smem(ra), s, ra);
    else
        launch_pdl(k_reduce<R, false>, (unsigned)(2 * ninst), kRedThreads, reduce_smem(ra), s,
                   ra);
}

int64_t serial_length(int64_t M, int64_t N, int64_t D) { return M * N + D * N - D; }

bool geometry(const semd_params &p, int64_t rows, int64_t cols, int order, int64_t &M,
              int64_t &N, int64_t &D, std::string &err)
{
    if (rows < 1 || cols < 1) {
        err = "rows and cols must be >= 1";
        return false;
    }
    M = order == SEMD_ORDER_ROWS ? cols : rows;
    N = order == SEMD_ORDER_ROWS ? rows : cols;
    D = p.transition_len < 0 ? (int64_t)std::llround(0.2 * (double)M) : p.transition_len;
    if (N == 1)
        D = 0; // one signal: there is nothing to join
    if (D > M) {
        err = "transition_len must be <= M (X_A needs D rows, Sec. 3.2)";
        return false;
    }
    if (serial_length(M, N, D) >= (int64_t)1 << 30) {
        err = "serialized length must be < 2^30";
        return false;
    }
    return true;
}

bool validate(const semd_params &p, std::string &err)
{
    if (p.order != SEMD_ORDER_ROWS && p.order != SEMD_ORDER_COLS)
        return err = "order must be ROWS or COLS", false;
    if (p.max_imfs < 1 || p.max_imfs > KMAX)
        return err = "max_imfs must be in [1, 32]", false;
    if (p.stop != SEMD_STOP_FIXED && p.stop != SEMD_STOP_SD && p.stop != SEMD_STOP_SNUMBER)
        return err = "stop must be FIXED, SD or SNUMBER", false;
    if (p.stop == SEMD_STOP_FIXED && (p.fixed_sifts < 1 || p.fixed_sifts > 1000))
        return err = "fixed_sifts must be in [1, 1000]", false;
    if (p.stop == SEMD_STOP_SD && (p.max_sifts < 1 || p.max_sifts > 1000 || !(p.sd_threshold >= 0)))
        return err = "max_sifts must be in [1, 1000] and sd_threshold >= 0", false;
    if (p.stop == SEMD_STOP_SNUMBER &&
        (p.max_sifts < 1 || p.max_sifts > 1000 || p.s_number < 1 || p.s_number > 1000))
        return err = "max_sifts and s_number must be in [1, 1000]", false;
    if (p.boundary != SEMD_BOUNDARY_MIRROR && p.boundary != SEMD_BOUNDARY_ENDPOINTS)
        return err = "boundary must be MIRROR or ENDPOINTS", false;
    if (p.boundary == SEMD_BOUNDARY_MIRROR && (p.mirror_knots < 1 || p.mirror_knots > 2))
        return err = "mirror_knots must be 1 or 2", false;
    if (p.precision != SEMD_FP64 && p.precision != SEMD_FP32_MIXED)
        return err = "precision must be FP64 or FP32_MIXED", false;
    if (p.spline_end != SEMD_SPLINE_NATURAL && p.spline_end != SEMD_SPLINE_NOT_A_KNOT)
        return err = "spline_end must be NATURAL or NOT_A_KNOT", false;
    if (p.ensemble_trials > 1 && !(p.noise_rel_std >= 0))
        return err = "noise_rel_std must be >= 0", false;
    if (p.transition_len < -1)
        return err = "transition_len must be >= -1", false;
    return true;
}

// Tile of the pass kernel for a plan: 1024 samples (128 threads).
// The plan's pass-kernel shape: the tuning table's entry for the plan's key when there is
// one, else 256-sample tiles and as many CTAs per SM as fit.
void choose_pass_shape(const semd_params &p, int64_t L, int ninst, int &tile, int &ctas,
                       int &variant)
{
    tile = kTile;
    ctas = 0;
    variant = 0;
    tune_lookup(p, L, ninst, tile, ctas, variant);
}

int max_iterations(const semd_params &p)
{
    return p.stop == SEMD_STOP_FIXED ? 1 + p.max_imfs * p.fixed_sifts
                                     : 1 + p.max_imfs * (p.max_sifts + 1);
}

#define SEMD_CU(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return SEMD_ECUDA;                                                             \
        }                                                                                  \
    } while (0)

semd_status Workspace::allocate(int64_t samples, int insts, int64_t tiles, int64_t rentries,
                                int iters, size_t elem, int64_t eemd_elems, size_t budget,
                                std::string &err)
{
    cap_samples = samples;
    cap_inst = insts;
    cap_tiles = tiles;
    cap_rentries = rentries;
    cap_iters = iters;
    elem_size = elem;
    struct Req {
        void **p;
        size_t bytes;
    };
    std::vector<Req> reqs = {
        {&h0, (size_t)samples * elem},
        {&h1, (size_t)samples * elem},
        {(void **)&r0, (size_t)samples * 8},
        {(void **)&r1, (size_t)samples * 8},
        {(void **)&d_inst, (size_t)insts * sizeof(Inst)},
        {(void **)&d_state, (size_t)insts * sizeof(State)},
        {(void **)&d_tile_inst, (size_t)tiles * 4},
        {&d_tex, (size_t)tiles * 2 * tile_rec_bytes(elem)},
        {(void **)&d_tsol, (size_t)tiles * 2 * sizeof(TileSolve)},
        {(void **)&d_taux, (size_t)tiles * sizeof(TileAux)},
        {(void **)&d_kmask, (size_t)tiles * 32 * sizeof(uint2)},
        {(void **)&d_rscr, (size_t)rentries * 8},
        {(void **)&d_active, (size_t)(iters + 8) * 4},
        {(void **)&d_beta, (size_t)(1 + 2 * kStdBlocks) * 8},
        {(void **)&d_misc, (size_t)tiles * 2 * 4 + 64},
        {(void **)&d_stats, sizeof(Stats)},
    };
    if (eemd_elems > 0) {
        reqs.push_back({&eemd_scratch, (size_t)eemd_elems * elem});
        reqs.push_back({(void **)&d_ce, sizeof(CeArgs)});
        reqs.push_back({(void **)&d_cestate, sizeof(CeState)});
        reqs.push_back({(void **)&d_cecount, (size_t)insts * 4});
        reqs.push_back({(void **)&d_ce_r, (size_t)(samples / insts) * 8});
        reqs.push_back({(void **)&d_cepart,
                        (size_t)((samples / insts + kCeTestSpan - 1) / kCeTestSpan + 1) *
                            sizeof(CePart)});
    }
    size_t total = 0;
    for (auto &r : reqs)
        total += (r.bytes + 255) & ~(size_t)255;
    if (budget > 0 && total > budget) {
        err = "workspace of " + std::to_string(total) + " bytes exceeds the budget of " +
              std::to_string(budget);
        return SEMD_EBUDGET;
    }
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc of the workspace: ") + cudaGetErrorString(e);
        (void)cudaGetLastError(); // a failed allocation must not surface in later calls
        base = nullptr;
        return e == cudaErrorMemoryAllocation ? SEMD_ENOMEM : SEMD_ECUDA;
    }
    bytes = total;
    char *cur = (char *)base;
    for (auto &r : reqs) {
        *r.p = cur;
        cur += (r.bytes + 255) & ~(size_t)255;
    }
    e = cudaMallocHost((void **)&h_inst, (size_t)insts * sizeof(Inst));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&h_tile_inst, (size_t)tiles * 4);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&h_state, (size_t)insts * sizeof(State));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&h_misc, (size_t)tiles * 2 * 4 + 64);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&h_stats, sizeof(Stats));
    if (e == cudaSuccess && eemd_elems > 0)
        e = cudaMallocHost((void **)&h_ce, sizeof(CeArgs));
    if (e == cudaSuccess && eemd_elems > 0)
        e = cudaMallocHost((void **)&h_cestate, sizeof(CeState));
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&staging_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        err = std::string("pinned host staging: ") + cudaGetErrorString(e);
        return SEMD_ENOMEM;
    }
    if (elem == 8)
        e = set_smem_attr<double>();
    else
        e = set_smem_attr<float>();
    if (e != cudaSuccess) {
        err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return SEMD_ECUDA;
    }
    return SEMD_OK;
}

void Workspace::release()
{
    if (staging_done) {
        cudaEventSynchronize(staging_done);
        cudaEventDestroy(staging_done);
    }
    if (base)
        cudaFree(base);
    if (h_inst)
        cudaFreeHost(h_inst);
    if (h_tile_inst)
        cudaFreeHost(h_tile_inst);
    if (h_state)
        cudaFreeHost(h_state);
    if (h_misc)
        cudaFreeHost(h_misc);
    if (h_stats)
        cudaFreeHost(h_stats);
    if (h_ce)
        cudaFreeHost(h_ce);
    if (h_cestate)
        cudaFreeHost(h_cestate);
    *this = Workspace();
}

// Points instance i at its own slices of the workspace buffers (samples from `off`,
// tiles from `tiles`, interface scratch from double `rent`).
static void bind_instance(Workspace &ws, Inst &in, int64_t off, int64_t tiles, int64_t rent)
{
    in.tile0 = (int32_t)tiles;
    in.ntiles = (int32_t)((in.L + ws.tile - 1) / ws.tile);
    in.h[0] = (char *)ws.h0 + off * (int64_t)ws.elem_size;
    in.h[1] = (char *)ws.h1 + off * (int64_t)ws.elem_size;
    in.r[0] = ws.r0 + off;
    in.r[1] = ws.r1 + off;
    in.tex = (char *)ws.d_tex + 2 * tiles * (int64_t)tile_rec_bytes(ws.elem_size);
    in.tsol = ws.d_tsol + 2 * tiles;
    in.taux = ws.d_taux + tiles;
    in.kmask = ws.d_kmask + 32 * tiles;
    in.rlen = reduce_len(in.ntiles);
    in.rscr = ws.d_rscr + rent;
}

// Lays out n instances (host descriptors in ws.h_inst must have L, geometry and output
// pointers set): buffer slices, tiles, then the upload of descriptors and tile map.
semd_status Workspace::layout(int n, int64_t &ntiles, cudaStream_t s, std::string &err)
{
    int64_t off = 0, tiles = 0, rent = 0;
    max_ntiles = 0;
    min_ntiles = INT64_MAX;
    for (int i = 0; i < n; ++i) {
        Inst &in = h_inst[i];
        bind_instance(*this, in, off, tiles, rent);
        off += (in.L + 31) & ~(int64_t)31;
        tiles += in.ntiles;
        rent += 2 * rscr_env_doubles(in.rlen);
        max_ntiles = std::max<int64_t>(max_ntiles, in.ntiles);
        min_ntiles = std::min<int64_t>(min_ntiles, in.ntiles);
    }
    if (off > cap_samples || tiles > cap_tiles || rent > cap_rentries || n > cap_inst) {
        err = "batch exceeds the plan's capacity";
        return SEMD_EBUDGET;
    }
    for (int i = 0; i < n; ++i)
        for (int t = 0; t < h_inst[i].ntiles; ++t)
            h_tile_inst[h_inst[i].tile0 + t] = i;
    ntiles = tiles;
    SEMD_CU(cudaMemcpyAsync(d_inst, h_inst, (size_t)n * sizeof(Inst), cudaMemcpyHostToDevice, s));
    SEMD_CU(cudaMemcpyAsync(d_tile_inst, h_tile_inst, (size_t)tiles * 4, cudaMemcpyHostToDevice,
                            s));
    SEMD_CU(cudaEventRecord(staging_done, s));
    return SEMD_OK;
}

template <typename R>
static void launch_pass(Workspace &ws, int64_t ntiles, bool need_sd, bool need_zc,
                        cudaStream_t s)
{
    PassArgs pa;
    pa.inst = ws.d_inst;
    pa.state = ws.d_state;
    pa.tile_inst = ws.d_tile_inst;
    pa.ntiles = ntiles;
    pa.need_sd = need_sd ? 1 : 0;
    pa.need_zc = need_zc ? 1 : 0;
    launch_pass_tiles<R>(ws.tile, ws.pass_variant, ws.pass_ctas, pa, ntiles, s);
}

// Shape of the interface solve of a launch whose instances have min_nt..max_nt tiles.
// An instance whose system fits in one CTA's shared memory is solved by one CTA per
// envelope. A longer one (natural spline ends) by a cluster of CLd CTAs per envelope, CLd
// the largest size of 16 or 8 the device can hold at full shared memory, while a CTA's
// share of its system fits; longer ones again by one CTA with a global-memory scratch.
template <typename R>
static void set_reduce_shape_t(ReduceArgs &ra, int64_t min_nt, int64_t max_nt)
{
    auto fits_one = [](int64_t nt) {
        return reduce_smem_bytes(reduce_len(nt), sizeof(R)) <= kReduceSmemMax;
    };
    ra.cl = 0;
    ra.cl_entries = 0;
    ra.cl_min_nt = ra.cl_max_nt = 0;
    ra.run_cl = 0;
    ra.run_single = 1;
    const int CLd = cluster_fits<R>(16, kClSmemOptin) ? 16 : cluster_fits<R>(8, kClSmemOptin) ? 8 : 0;
    if (CLd > 0 && ra.spline_end == SPLINE_NATURAL) {
        int64_t lo = 1;
        while (fits_one(lo * 2))
            lo *= 2;
        int64_t hi = lo * 2; // fits_one(lo), !fits_one(hi): the boundary in between
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) / 2;
            (fits_one(mid) ? lo : hi) = mid;
        }
        int64_t top = hi; // the largest count whose cluster share fits
        while (cl_smem_bytes<R>(cl_entries((top * 2 + CLd - 1) / CLd)) <= kClSmemOptin - 1024)
            top *= 2;
        int64_t b = top * 2;
        while (b - top > 1) {
            const int64_t mid = (top + b) / 2;
            (cl_smem_bytes<R>(cl_entries((mid + CLd - 1) / CLd)) <= kClSmemOptin - 1024 ? top : b) = mid;
        }
        if (top >= hi && top < (int64_t)1 << 30) {
            ra.cl = CLd;
            ra.cl_min_nt = (int32_t)hi;
            ra.cl_max_nt = (int32_t)top;
        }
    }
    if (ra.cl > 0) {
        ra.run_cl = (max_nt >= ra.cl_min_nt && min_nt <= ra.cl_max_nt) ? 1 : 0;
        ra.run_single = (min_nt < ra.cl_min_nt || max_nt > ra.cl_max_nt) ? 1 : 0;
        const int64_t mc = std::min<int64_t>(max_nt, ra.cl_max_nt);
        ra.cl_entries = cl_entries((mc + ra.cl - 1) / ra.cl);
        // the one-CTA kernel's instances: below cl_min_nt (shared memory), or beyond
        // cl_max_nt (global memory)
        const int64_t ms = max_nt > ra.cl_max_nt ? max_nt : std::min<int64_t>(max_nt, ra.cl_min_nt - 1);
        ra.smem_entries = fits_one(ms) ? reduce_len(ms) : 0;
    } else {
        ra.smem_entries = fits_one(max_nt) ? reduce_len(max_nt) : 0;
    }
}
static void set_reduce_shape(ReduceArgs &ra, int64_t min_nt, int64_t max_nt, size_t elem)
{
    if (elem == 8)
        set_reduce_shape_t<double>(ra, min_nt, max_nt);
    else
        set_reduce_shape_t<float>(ra, min_nt, max_nt);
}

static ReduceArgs reduce_args(Workspace &ws, const semd_params &p)
{
    ReduceArgs ra;
    ra.inst = ws.d_inst;
    ra.state = ws.d_state;
    ra.inst_list = nullptr;
    ra.active = ws.d_active;
    ra.stats = ws.d_stats;
    ra.K = p.max_imfs;
    ra.stop = p.stop;
    ra.fixed_sifts = p.fixed_sifts;
    ra.max_sifts = p.max_sifts;
    ra.sd_threshold = p.sd_threshold;
    ra.boundary = p.boundary;
    ra.mirror_knots = p.mirror_knots;
    ra.single = ws.elem_size == 4 ? 1 : 0;
    ra.s_number = p.s_number;
    ra.spline_end = p.spline_end;
    set_reduce_shape(ra, ws.min_ntiles, ws.max_ntiles, ws.elem_size);
    return ra;
}

// Records an event pair around a launch when the plan is profiling.
struct LaunchTimer {
    Profiler *pr;
    cudaStream_t s;
    int kind; // 0 pass, 1 reduce
    size_t slot = 0;
    LaunchTimer(Profiler *p, cudaStream_t st, int k) : pr(p), s(st), kind(k)
    {
        if (pr && pr->on)
            slot = pr->begin(kind, s);
    }
    ~LaunchTimer()
    {
        if (pr && pr->on)
            pr->end(slot, s);
    }
};

// Iterations of the body of a device-decided sifting loop.
constexpr int kLoopBody = 4;

// End of one body execution of a device-decided sifting loop (Sec. 2.1 Step 5 with an
// adaptive stop rule): the loop goes on while the body's last interface solve counted a
// running instance and the iteration cap is not reached. Clears the body's counters for
// its next execution.
__global__ void k_loop_control(cudaGraphConditionalHandle h, int32_t *active, int32_t *iter,
                               int max_iters)
{
    const int it = *iter + kLoopBody;
    const bool more = active[kLoopBody - 1] > 0 && it < max_iters;
    *iter = it;
    for (int b = 0; b < kLoopBody; ++b)
        active[b] = 0;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// The sifting passes of one decomposition: `iters` pass + interface-solve launches (the
// state machine idles finished instances). With an adaptive stop rule (SD, S-number):
// under capture, a WHILE conditional node whose body runs kLoopBody iterations and then
// decides on the device whether to go on (no host synchronization); without capture,
// every eighth iteration reads the count of running instances and ends the loop at zero.
template <typename R>
static semd_status sift_loop(semd_plan_s &pl, ReduceArgs ra, int ninst, int64_t ntiles,
                             int iters, cudaStream_t s, Profiler *prof, bool capture,
                             int64_t &launches)
{
    Workspace &ws = pl.ws;
    std::string &err = pl.err;
    const bool sd = ra.stop == SEMD_STOP_SD, zc = ra.stop == SEMD_STOP_SNUMBER;
    if (capture && (sd || zc)) {
        cudaStreamCaptureStatus cs;
        unsigned long long id = 0;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *ed = nullptr;
        size_t nd = 0;
        SEMD_CU(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &ed, &nd));
        cudaGraphConditionalHandle h;
        SEMD_CU(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t cn;
        SEMD_CU(cudaGraphAddNode(&cn, g, deps, ed, nd, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        SEMD_CU(cudaStreamBeginCaptureToGraph(pl.lstream, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
        g_plain_launches = true;
        for (int b = 0; b < kLoopBody; ++b) {
            launch_pass<R>(ws, ntiles, sd, zc, pl.lstream);
            ra.active = ws.d_active + b;
            launch_reduce<R>(ra, ninst, pl.lstream);
        }
        g_plain_launches = false;
        k_loop_control<<<1, 1, 0, pl.lstream>>>(h, ws.d_active, ws.d_active + kLoopBody, iters);
        cudaGraph_t bo = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(pl.lstream, &bo);
        SEMD_CU(ce);
        SEMD_CU(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies));
        launches += 2 * kLoopBody + 1; // per body execution
        return SEMD_OK;
    }
    for (int it = 0; it < iters; ++it) {
        {
            LaunchTimer t(prof, s, 0);
            launch_pass<R>(ws, ntiles, sd, zc, s);
        }
        ra.active = ws.d_active + it;
        {
            LaunchTimer t(prof, s, 1);
            launch_reduce<R>(ra, ninst, s);
        }
        launches += 2;
        if (!capture && (sd || zc) && (it % 8) == 7) {
            SEMD_CU(cudaMemcpyAsync(ws.h_misc, ws.d_active + it, 4, cudaMemcpyDeviceToHost, s));
            SEMD_CU(cudaStreamSynchronize(s));
            if (((int32_t *)ws.h_misc)[0] == 0)
                break;
        }
    }
    return SEMD_OK;
}

// All device work of one decomposition after the descriptors are uploaded. Everything
// here is stream-ordered and, for the fixed sift count, free of host synchronization,
// so it can be captured into a CUDA graph.
template <typename R>
static semd_status enqueue_decomposition(semd_plan_s &pl, int ninst, int64_t ntiles,
                                         int ntiles0, cudaStream_t s, bool capture)
{
    Workspace &ws = pl.ws;
    std::string &err = pl.err;
    const semd_params &p = pl.p;
    const bool eemd = p.ensemble_trials > 1;
    Profiler *prof = capture ? nullptr : &pl.prof;
    int64_t launches = 0;
    const int iters = max_iterations(p);
    SEMD_CU(cudaMemsetAsync(ws.d_state, 0, (size_t)ninst * sizeof(State), s));
    SEMD_CU(cudaMemsetAsync(ws.d_active, 0, (size_t)(iters + kLoopBody + 1) * 4, s));
    SEMD_CU(cudaMemsetAsync(ws.d_stats, 0, sizeof(Stats), s));
    k_serialize<R><<<(unsigned)ntiles, 256, 0, s>>>(ws.d_inst, ws.d_state, ws.d_tile_inst,
                                                      ws.tile, eemd ? 1 : 0);
    ++launches;
    if (eemd) {
        for (int stage = 0; stage < 3; ++stage)
            k_std<<<stage == 2 ? 1 : kStdBlocks, kStdThreads, 0, s>>>(
                ws.d_inst, p.noise_rel_std, ws.d_beta, ws.d_beta + 1, stage);
        for (int m0 = 1; m0 < ninst; m0 += 65535) { // grid y is at most 65535
            k_add_noise<R><<<noise_grid(ntiles0, ws.tile, std::min(ninst - m0, 65535)), 256, 0,
                             s>>>(ws.d_inst, m0, ws.d_beta, pl.noise_seed);
            ++launches;
        }
        k_add_noise<R><<<noise_grid(ntiles0, ws.tile, 1), 256, 0, s>>>(ws.d_inst, 0, ws.d_beta,
                                                                      pl.noise_seed);
        launches += 4;
    }
    ReduceArgs ra = reduce_args(ws, p);
    semd_status st = sift_loop<R>(pl, ra, ninst, ntiles, iters, s, prof, capture, launches);
    if (st != SEMD_OK)
        return st;
    if (eemd) {
        const int64_t L0 = (int64_t)ntiles0 * ws.tile; // at least the signal's length
        const dim3 ag((unsigned)((L0 + 256 * kAvgPer - 1) / (256 * kAvgPer)),
                      (unsigned)(p.max_imfs + 1));
        k_eemd_average<R><<<ag, 256, 0, s>>>(ws.d_inst, ws.d_state, ninst, p.max_imfs,
                                             (const R *)ws.eemd_scratch);
    } else {
        k_finalize<R><<<(unsigned)ntiles, 256, 0, s>>>(ws.d_inst, ws.d_state, ws.d_tile_inst,
                                                         ws.tile, p.max_imfs);
    }
    ++launches;
    SEMD_CU(cudaGetLastError());
    pl.stat_launches = launches;
    return SEMD_OK;
}

template <typename R>
semd_status decompose_impl(semd_plan_s &pl, int count, const semd_instance *insts,
                           const void *d_noise, int *n_imfs, cudaStream_t s,
                           int64_t imf_stride_all)
{
    NvtxRange nvtx("serial_emd_decompose");
    Workspace &ws = pl.ws;
    std::string &err = pl.err;
    const semd_params &p = pl.p;
    const bool eemd = p.ensemble_trials > 1;
    const int ninst = eemd ? p.ensemble_trials : count;
    SEMD_CU(cudaEventSynchronize(ws.staging_done)); // staging buffers are free again
    for (int i = 0; i < ninst; ++i) {
        const semd_instance &q = insts[eemd ? 0 : i];
        Inst in{};
        int64_t M, N, D;
        if (!geometry(p, q.rows, q.cols, p.order, M, N, D, err))
            return SEMD_EINVAL;
        in.L = serial_length(M, N, D);
        in.M = M;
        in.N = N;
        in.D = D;
        in.order = p.order;
        in.x = q.d_x;
        if (eemd) {
            const int64_t slot = (in.L + 31) & ~(int64_t)31; // keeps every slot 128-byte aligned
            in.imf = (char *)ws.eemd_scratch + (size_t)i * p.max_imfs * slot * sizeof(R);
            in.imf_stride = slot;
            in.imf_serialized = 1;
            in.res = nullptr;
            if (i == 0) {
                in.noise = d_noise;
                in.avg_imf = q.d_imfs;
                in.avg_res = q.d_residue;
            }
        } else {
            in.imf = q.d_imfs;
            in.imf_stride = imf_stride_all > 0 ? imf_stride_all : q.rows * q.cols;
            in.imf_serialized = 0;
            in.res = q.d_residue;
        }
        ws.h_inst[i] = in;
    }
    int64_t ntiles;
    semd_status st = ws.layout(ninst, ntiles, s, err);
    if (st != SEMD_OK)
        return st;
    const int ntiles0 = ws.h_inst[0].ntiles;
    const bool use_graph = pl.graphs && !pl.prof.on;
    pl.prof.reset();
    if (use_graph) {
        const GraphKey key{ninst,         ntiles,         ntiles0,        ws.max_ntiles, ws.tile,
                           ws.pass_ctas,  ws.pass_variant, pl.noise_seed, ws.min_ntiles};
        if (!pl.graph_exec || !(pl.graph_key == key)) {
            if (pl.graph_exec) {
                cudaGraphExecDestroy(pl.graph_exec);
                pl.graph_exec = nullptr;
            }
            // capture on the plan's own stream so that any caller stream (including the
            // legacy default stream) can be used
            cudaGraph_t g = nullptr;
            SEMD_CU(cudaStreamBeginCapture(pl.gstream, cudaStreamCaptureModeThreadLocal));
            st = enqueue_decomposition<R>(pl, ninst, ntiles, ntiles0, pl.gstream, true);
            cudaError_t ce = cudaStreamEndCapture(pl.gstream, &g);
            if (st != SEMD_OK) {
                if (g)
                    cudaGraphDestroy(g);
                return st;
            }
            SEMD_CU(ce);
            ce = cudaGraphInstantiate(&pl.graph_exec, g, 0);
            cudaGraphDestroy(g);
            SEMD_CU(ce);
            pl.graph_key = key;
            pl.graph_launches = pl.stat_launches;
        }
        SEMD_CU(cudaEventRecord(pl.ev_in, s));
        SEMD_CU(cudaStreamWaitEvent(pl.gstream, pl.ev_in, 0));
        SEMD_CU(cudaGraphLaunch(pl.graph_exec, pl.gstream));
        SEMD_CU(cudaEventRecord(pl.ev_out, pl.gstream));
        SEMD_CU(cudaStreamWaitEvent(s, pl.ev_out, 0));
        pl.stat_launches = pl.graph_launches;
        pl.stat_graph = 1;
    } else {
        st = enqueue_decomposition<R>(pl, ninst, ntiles, ntiles0, s, false);
        if (st != SEMD_OK)
            return st;
        pl.stat_graph = 0;
    }
    SEMD_CU(cudaMemcpyAsync(ws.h_state, ws.d_state, (size_t)ninst * sizeof(State),
                            cudaMemcpyDeviceToHost, s));
    SEMD_CU(cudaMemcpyAsync(ws.h_stats, ws.d_stats, sizeof(Stats), cudaMemcpyDeviceToHost, s));
    pl.last_ninst = ninst;
    pl.last_count = eemd ? 1 : count;
    pl.last_ceemdan = false;
    if (n_imfs) {
        SEMD_CU(cudaStreamSynchronize(s));
        pl.counts(pl.last_count, n_imfs, nullptr);
    }
    return SEMD_OK;
}

// All device work of one CEEMDAN call (Sec. 2.2, Steps 1-4) after the descriptors and
// the call's arguments are uploaded: the EMD of the noise realizations, then K stages.
// Stream-ordered and, for the fixed sift count, free of host synchronization.
template <typename R>
static semd_status enqueue_ceemdan(semd_plan_s &pl, int64_t ntiles, cudaStream_t s, bool capture)
{
    Workspace &ws = pl.ws;
    std::string &err = pl.err;
    const semd_params &p = pl.p;
    const int trials = p.ensemble_trials, K = p.max_imfs;
    Profiler *prof = capture ? nullptr : &pl.prof;
    int64_t launches = 0;
    const int64_t L = ws.h_ce->L;
    const unsigned eg = (unsigned)std::min<int64_t>((L + 255) / 256, 4 * 304);
    // stage test: one block per kCeTestSpan samples; stage inputs: one grid row per trial,
    // about 4 x 152 blocks in all; average: one block per 32 samples
    const unsigned tg = (unsigned)((L + kCeTestSpan - 1) / kCeTestSpan);
    const unsigned ig = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((L + 255) / 256, (4 * 152 + trials - 1) / trials));
    const unsigned ag = (unsigned)((L + 31) / 32);
    SEMD_CU(cudaMemsetAsync(ws.d_stats, 0, sizeof(Stats), s));
    ReduceArgs ra = reduce_args(ws, p);
    semd_status st;
    if (K >= 2) { // E_1 .. E_{K-1} of every realization: plain EMD with K-1 IMFs
        semd_params pn = p;
        pn.max_imfs = K - 1;
        const int iters = max_iterations(pn);
        SEMD_CU(cudaMemsetAsync(ws.d_state, 0, (size_t)trials * sizeof(State), s));
        SEMD_CU(cudaMemsetAsync(ws.d_active, 0, (size_t)(iters + kLoopBody + 1) * 4, s));
        k_serialize<R><<<(unsigned)ntiles, 256, 0, s>>>(ws.d_inst, ws.d_state, ws.d_tile_inst,
                                                          ws.tile, 0);
        ++launches;
        ra.K = K - 1;
        st = sift_loop<R>(pl, ra, trials, ntiles, iters, s, prof, capture, launches);
        if (st != SEMD_OK)
            return st;
    }
    k_ce_setup<<<1, 256, 0, s>>>(ws.d_ce, ws.d_inst, ws.d_state, ws.d_cestate, K >= 2 ? 1 : 0,
                                 (int)sizeof(R));
    k_ce_serialize<R><<<eg, 256, 0, s>>>(ws.d_ce);
    launches += 2;
    semd_params p1 = p;
    p1.max_imfs = 1;
    const int iters1 = max_iterations(p1);
    ra.K = 1;
    for (int k = 0; k < K; ++k) {
        NvtxRange stage_range("ceemdan stage");
        k_ce_stage_test<<<tg, 256, 0, s>>>(ws.d_ce, ws.d_cestate, ws.d_cepart, 0);
        k_ce_stage_test<<<tg, 256, 0, s>>>(ws.d_ce, ws.d_cestate, ws.d_cepart, 1);
        SEMD_CU(cudaMemsetAsync(ws.d_state, 0, (size_t)trials * sizeof(State), s));
        SEMD_CU(cudaMemsetAsync(ws.d_active, 0, (size_t)(iters1 + kLoopBody + 1) * 4, s));
        k_ce_stage_init<R><<<dim3(ig, (unsigned)trials), 256, 0, s>>>(ws.d_ce, ws.d_inst,
                                                                      ws.d_state, ws.d_cestate,
                                                                      k);
        launches += 3;
        st = sift_loop<R>(pl, ra, trials, ntiles, iters1, s, prof, capture, launches);
        if (st != SEMD_OK)
            return st;
        k_ce_average<R><<<ag, 32 * kCeAvgGroups, 0, s>>>(ws.d_ce, ws.d_inst, ws.d_state, k);
        ++launches;
    }
    k_ce_finish<<<eg, 256, 0, s>>>(ws.d_ce);
    ++launches;
    SEMD_CU(cudaGetLastError());
    pl.stat_launches = launches;
    return SEMD_OK;
}

template <typename R>
semd_status ceemdan_impl(semd_plan_s &pl, const void *d_x, const void *d_noise, void *d_modes,
                         double *d_residue, int *n_imfs, cudaStream_t s)
{
    NvtxRange nvtx("serial_emd_ceemdan");
    Workspace &ws = pl.ws;
    std::string &err = pl.err;
    const semd_params &p = pl.p;
    const int trials = p.ensemble_trials, K = p.max_imfs;
    SEMD_CU(cudaEventSynchronize(ws.staging_done)); // staging buffers are free again
    int64_t M, N, D;
    if (!geometry(p, p.rows, p.cols, p.order, M, N, D, err))
        return SEMD_EINVAL;
    const int64_t L = serial_length(M, N, D);
    const int64_t slot = (L + 31) & ~(int64_t)31;
    // the trials, first as the EMD of the noise realizations (one plain signal each)
    for (int m = 0; m < trials; ++m) {
        Inst in{};
        in.L = L;
        in.M = L;
        in.N = 1;
        in.D = 0;
        in.order = 0;
        in.x = (const char *)d_noise + (size_t)m * (size_t)L * sizeof(R);
        in.imf = (char *)ws.eemd_scratch + (size_t)m * K * slot * sizeof(R);
        in.imf_stride = slot;
        in.imf_serialized = 1;
        in.res = nullptr;
        ws.h_inst[m] = in;
    }
    CeArgs &a = *ws.h_ce;
    a = CeArgs{};
    a.x = d_x;
    a.noise = d_noise;
    a.E = ws.eemd_scratch;
    a.modes = d_modes;
    a.res = d_residue;
    a.r = ws.d_ce_r;
    a.ncount = ws.d_cecount;
    a.M = M;
    a.N = N;
    a.D = D;
    a.L = L;
    a.slot = slot;
    a.order = p.order;
    a.trials = trials;
    a.K = K;
    a.rel = p.noise_rel_std;
    SEMD_CU(cudaMemcpyAsync(ws.d_ce, ws.h_ce, sizeof(CeArgs), cudaMemcpyHostToDevice, s));
    int64_t ntiles;
    semd_status st = ws.layout(trials, ntiles, s, err); // records staging_done
    if (st != SEMD_OK)
        return st;
    const bool use_graph = pl.graphs && !pl.prof.on;
    pl.prof.reset();
    if (use_graph) {
        const GraphKey key{trials,       ntiles,          ws.h_inst[0].ntiles, ws.max_ntiles,
                           ws.tile,      ws.pass_ctas,    ws.pass_variant,     0,
                           ws.min_ntiles};
        if (!pl.ce_graph_exec || !(pl.ce_graph_key == key)) {
            if (pl.ce_graph_exec) {
                cudaGraphExecDestroy(pl.ce_graph_exec);
                pl.ce_graph_exec = nullptr;
            }
            cudaGraph_t g = nullptr;
            SEMD_CU(cudaStreamBeginCapture(pl.gstream, cudaStreamCaptureModeThreadLocal));
            st = enqueue_ceemdan<R>(pl, ntiles, pl.gstream, true);
            cudaError_t ce = cudaStreamEndCapture(pl.gstream, &g);
            if (st != SEMD_OK) {
                if (g)
                    cudaGraphDestroy(g);
                return st;
            }
            SEMD_CU(ce);
            ce = cudaGraphInstantiate(&pl.ce_graph_exec, g, 0);
            cudaGraphDestroy(g);
            SEMD_CU(ce);
            pl.ce_graph_key = key;
            pl.ce_graph_launches = pl.stat_launches;
        }
        SEMD_CU(cudaEventRecord(pl.ev_in, s));
        SEMD_CU(cudaStreamWaitEvent(pl.gstream, pl.ev_in, 0));
        SEMD_CU(cudaGraphLaunch(pl.ce_graph_exec, pl.gstream));
        SEMD_CU(cudaEventRecord(pl.ev_out, pl.gstream));
        SEMD_CU(cudaStreamWaitEvent(s, pl.ev_out, 0));
        pl.stat_launches = pl.ce_graph_launches;
        pl.stat_graph = 1;
    } else {
        st = enqueue_ceemdan<R>(pl, ntiles, s, false);
        if (st != SEMD_OK)
            return st;
        pl.stat_graph = 0;
    }
    SEMD_CU(cudaMemcpyAsync(ws.h_cestate, ws.d_cestate, sizeof(CeState), cudaMemcpyDeviceToHost,
                            s));
    SEMD_CU(cudaMemcpyAsync(ws.h_stats, ws.d_stats, sizeof(Stats), cudaMemcpyDeviceToHost, s));
    pl.last_ninst = trials;
    pl.last_count = 1;
    pl.last_ceemdan = true;
    if (n_imfs) {
        SEMD_CU(cudaStreamSynchronize(s));
        *n_imfs = ws.h_cestate->n;
    }
    return SEMD_OK;
}

template <typename R>
semd_status extrema_impl(semd_plan_s &pl, const void *d_h, int64_t L, int32_t *tmax,
                         int32_t *tmin, int64_t *nmax, int64_t *nmin, cudaStream_t s)
{
    Workspace &ws = pl.ws;
    std::string &err = pl.err;
    const int ntiles = (int)((L + ws.tile - 1) / ws.tile);
    if (L < 1 || ntiles > ws.cap_tiles) {
        err = "L out of range for this plan";
        return SEMD_EINVAL;
    }
    int32_t *d_cnt = ws.d_misc;
    k_extrema_tiles<R><<<ntiles, 32, 0, s>>>((const R *)d_h, L, ws.tile, nullptr, d_cnt, nullptr,
                                             nullptr);
    SEMD_CU(cudaMemcpyAsync(ws.h_misc, d_cnt, (size_t)ntiles * 8, cudaMemcpyDeviceToHost, s));
    SEMD_CU(cudaStreamSynchronize(s));
    int32_t *c = (int32_t *)ws.h_misc;
    int64_t a = 0, b = 0;
    for (int t = 0; t < ntiles; ++t) {
        const int32_t ca = c[2 * t], cb = c[2 * t + 1];
        c[2 * t] = (int32_t)a;
        c[2 * t + 1] = (int32_t)b;
        a += ca;
        b += cb;
    }
    SEMD_CU(cudaMemcpyAsync(d_cnt, ws.h_misc, (size_t)ntiles * 8, cudaMemcpyHostToDevice, s));
    k_extrema_tiles<R><<<ntiles, 32, 0, s>>>((const R *)d_h, L, ws.tile, d_cnt, nullptr, tmax,
                                             tmin);
    SEMD_CU(cudaGetLastError());
    SEMD_CU(cudaStreamSynchronize(s));
    *nmax = a;
    *nmin = b;
    return SEMD_OK;
}

template <typename R>
semd_status sift_impl(semd_plan_s &pl, const void *d_h, int64_t L, void *d_out, double *sd_num,
                      double *sd_den, cudaStream_t s)
{
    Workspace &ws = pl.ws;
    std::string &err = pl.err;
    if (L < 1 || L > ws.cap_samples) {
        err = "L out of range for this plan";
        return SEMD_EINVAL;
    }
    SEMD_CU(cudaEventSynchronize(ws.staging_done));
    Inst in{};
    in.L = L;
    in.M = L;
    in.N = 1;
    in.D = 0;
    ws.h_inst[0] = in;
    int64_t ntiles;
    semd_status st = ws.layout(1, ntiles, s, err);
    if (st != SEMD_OK)
        return st;
    SEMD_CU(cudaMemsetAsync(ws.d_state, 0, sizeof(State), s));
    k_to_double<R><<<152, 256, 0, s>>>((const R *)d_h, L, ws.r0);
    semd_params p = pl.p;
    p.stop = SEMD_STOP_FIXED;
    p.fixed_sifts = 1000; // stay in SIFT mode
    p.max_imfs = 1;
    ReduceArgs ra = reduce_args(ws, p);
    SEMD_CU(cudaMemsetAsync(ws.d_active, 0, 8, s));
    launch_pass<R>(ws, ntiles, true, false, s); // INIT: h = r, export
    launch_reduce<R>(ra, 1, s);
    launch_pass<R>(ws, ntiles, true, false, s); // SIFT
    SEMD_CU(cudaGetLastError());
    SEMD_CU(cudaMemcpyAsync(ws.h_state, ws.d_state, sizeof(State), cudaMemcpyDeviceToHost, s));
    SEMD_CU(cudaStreamSynchronize(s));
    if (ws.h_state[0].mode != MODE_SIFT) {
        err = "the signal lacks maxima or minima; it cannot be sifted";
        return SEMD_EINVAL;
    }
    // the SIFT pass read h from buffer hpar = 1 and wrote buffer 0
    SEMD_CU(cudaMemcpyAsync(d_out, ws.h0, (size_t)L * sizeof(R), cudaMemcpyDeviceToDevice, s));
    std::vector<TileAux> aux(ntiles);
    SEMD_CU(cudaMemcpyAsync(aux.data(), ws.d_taux, (size_t)ntiles * sizeof(TileAux),
                            cudaMemcpyDeviceToHost, s));
    SEMD_CU(cudaStreamSynchronize(s));
    double a = 0.0, b = 0.0;
    for (auto &x : aux) {
        a += x.sd_num;
        b += x.sd_den;
    }
    *sd_num = a;
    *sd_den = b;
    return SEMD_OK;
}

// ------------------------------------------------- launch helpers for other translation units

cudaError_t setup_kernel_attrs(size_t elem)
{
    return elem == 8 ? set_smem_attr<double>() : set_smem_attr<float>();
}

void launch_pass_any(size_t elem, int tile, const PassArgs &pa, int64_t ntiles, cudaStream_t s,
                     int ctas_per_sm)
{
    if (elem == 8)
        launch_pass_tiles<double>(tile, 0, ctas_per_sm, pa, ntiles, s);
    else
        launch_pass_tiles<float>(tile, 0, ctas_per_sm, pa, ntiles, s);
}

void launch_reduce_any(size_t elem, const ReduceArgs &ra, int nblocks, cudaStream_t s)
{
    if (elem == 8)
        launch_reduce<double>(ra, nblocks, s);
    else
        launch_reduce<float>(ra, nblocks, s);
}

void launch_serialize_any(size_t elem, const Inst *d_inst, const State *d_state,
                          const int32_t *tile_inst, int64_t ntiles, int tile, cudaStream_t s)
{
    if (elem == 8)
        k_serialize<double><<<(unsigned)ntiles, 256, 0, s>>>(d_inst, d_state, tile_inst, tile, 0);
    else
        k_serialize<float><<<(unsigned)ntiles, 256, 0, s>>>(d_inst, d_state, tile_inst, tile, 0);
}

void launch_finalize_any(size_t elem, const Inst *d_inst, const State *d_state,
                         const int32_t *tile_inst, int64_t ntiles, int tile, int K,
                         cudaStream_t s)
{
    if (elem == 8)
        k_finalize<double><<<(unsigned)ntiles, 256, 0, s>>>(d_inst, d_state, tile_inst, tile, K);
    else
        k_finalize<float><<<(unsigned)ntiles, 256, 0, s>>>(d_inst, d_state, tile_inst, tile, K);
}

ReduceArgs make_reduce_args(const semd_params &p, const Inst *d_inst, State *d_state,
                            const int32_t *inst_list, int32_t *active, size_t elem,
                            int64_t min_ntiles, int64_t max_ntiles)
{
    ReduceArgs ra;
    ra.inst = d_inst;
    ra.state = d_state;
    ra.inst_list = inst_list;
    ra.active = active;
    ra.stats = nullptr;
    ra.K = p.max_imfs;
    ra.stop = p.stop;
    ra.fixed_sifts = p.fixed_sifts;
    ra.max_sifts = p.max_sifts;
    ra.sd_threshold = p.sd_threshold;
    ra.boundary = p.boundary;
    ra.mirror_knots = p.mirror_knots;
    ra.single = elem == 4 ? 1 : 0;
    ra.s_number = p.s_number;
    ra.spline_end = p.spline_end;
    set_reduce_shape(ra, min_ntiles, max_ntiles, elem);
    return ra;
}

template semd_status decompose_impl<float>(semd_plan_s &, int, const semd_instance *,
                                           const void *, int *, cudaStream_t, int64_t);
template semd_status decompose_impl<double>(semd_plan_s &, int, const semd_instance *,
                                            const void *, int *, cudaStream_t, int64_t);

} // namespace semd

void semd_plan_s::counts(int count, int *n_imfs, int *sifts) const
{
    using namespace semd;
    const bool eemd = p.ensemble_trials > 1;
    for (int i = 0; i < count; ++i) {
        int n = 0;
        if (last_ceemdan) {
            n = ws.h_cestate->n;
        } else if (eemd) {
            for (int m = 0; m < last_ninst; ++m)
                n = std::max(n, (int)ws.h_state[m].imf_count);
        } else {
            n = ws.h_state[i].imf_count;
        }
        if (n_imfs)
            n_imfs[i] = n;
        if (sifts)
            for (int k = 0; k < p.max_imfs; ++k)
                sifts[(int64_t)i * p.max_imfs + k] =
                    (eemd || last_ceemdan) ? 0 : (k < n ? ws.h_state[i].sifts[k] : 0);
    }
}

// ======================================================================= C ABI
using namespace semd;

extern "C" {

void serial_emd_default_params(semd_params *p)
{
    std::memset(p, 0, sizeof(*p));
    p->rows = 1;
    p->cols = 1;
    p->order = SEMD_ORDER_ROWS;
    p->transition_len = -1;
    p->max_imfs = 10;
    p->stop = SEMD_STOP_FIXED;
    p->fixed_sifts = 10;
    p->max_sifts = 50;
    p->sd_threshold = 0.2;
    p->boundary = SEMD_BOUNDARY_MIRROR;
    p->mirror_knots = 2;
    p->precision = SEMD_FP32_MIXED;
    p->ensemble_trials = 1;
    p->noise_rel_std = 0.2;
    p->s_number = 4;
}

semd_status serial_emd_plan(const semd_params *params, int max_batch, size_t mem_budget,
                            semd_plan_t *out)
{
    std::string &err = g_plan_create_error;
    err.clear();
    if (!params || !out || max_batch < 1) {
        err = "null argument or max_batch < 1";
        return SEMD_EINVAL;
    }
    *out = nullptr;
    if (!validate(*params, err))
        return SEMD_EINVAL;
    int64_t M, N, D;
    if (!geometry(*params, params->rows, params->cols, params->order, M, N, D, err))
        return SEMD_EINVAL;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        err = "no CUDA device is available";
        return SEMD_ECUDA;
    }
    const bool eemd = params->ensemble_trials > 1;
    if (eemd && max_batch != 1) {
        err = "EEMD plans take one input (max_batch = 1)";
        return SEMD_EINVAL;
    }
    const int64_t L = serial_length(M, N, D);
    const int ninst = eemd ? params->ensemble_trials : max_batch;
    int tile, ctas, variant;
    choose_pass_shape(*params, L, ninst, tile, ctas, variant);
    // capacity for the smallest tile, so that the tile can be changed per plan
    const int64_t tiles_per = (L + kMinTile - 1) / kMinTile;
    const int64_t samples = (int64_t)ninst * ((L + 31) & ~(int64_t)31);
    const int64_t tiles = (int64_t)ninst * tiles_per;
    const int64_t rent = (int64_t)ninst * 2 * rscr_env_doubles(reduce_len(tiles_per));
    const size_t elem = params->precision == SEMD_FP64 ? 8 : 4;
    const int64_t eemd_elems =
        eemd ? (int64_t)ninst * params->max_imfs * ((L + 31) & ~(int64_t)31) : 0;
    semd_plan_s *pl = new (std::nothrow) semd_plan_s();
    if (!pl) {
        err = "out of host memory";
        return SEMD_ENOMEM;
    }
    pl->p = *params;
    pl->L = L;
    pl->ws.tile = tile;
    pl->ws.pass_ctas = ctas;
    pl->ws.pass_variant = variant;
    semd_status st = pl->ws.allocate(samples, ninst, tiles, rent, max_iterations(*params), elem,
                                      eemd_elems, mem_budget, err);
    if (st == SEMD_OK) {
        if (cudaStreamCreateWithFlags(&pl->gstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&pl->lstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            err = "stream or event creation failed";
            st = SEMD_ECUDA;
        }
    }
    if (st != SEMD_OK) {
        serial_emd_destroy(pl);
        return st;
    }
    *out = pl;
    return SEMD_OK;
}

size_t serial_emd_plan_bytes(semd_plan_t plan) { return plan ? plan->ws.bytes : 0; }

semd_status serial_emd_decompose(semd_plan_t plan, const void *d_x, const void *d_noise,
                                 void *d_imfs, double *d_residue, int *n_imfs, void *stream)
{
    if (!plan)
        return SEMD_EINVAL;
    if (!d_x || !d_imfs) {
        plan->err = "null input or output pointer";
        return SEMD_EINVAL;
    }
    semd_instance in{d_x, plan->p.rows, plan->p.cols, d_imfs, d_residue};
    cudaStream_t s = (cudaStream_t)stream;
    return plan->p.precision == SEMD_FP64
               ? decompose_impl<double>(*plan, 1, &in, d_noise, n_imfs, s, 0)
               : decompose_impl<float>(*plan, 1, &in, d_noise, n_imfs, s, 0);
}

semd_status serial_emd_decompose_batch(semd_plan_t plan, int count, const semd_instance *inst,
                                       int *n_imfs, void *stream)
{
    if (!plan)
        return SEMD_EINVAL;
    if (plan->p.ensemble_trials > 1) {
        plan->err = "batched decomposition takes EMD plans only";
        return SEMD_EINVAL;
    }
    if (count < 1 || count > plan->ws.cap_inst || !inst) {
        plan->err = "count must be in [1, max_batch]";
        return SEMD_EINVAL;
    }
    const int64_t Lp = plan->L;
    for (int i = 0; i < count; ++i) {
        int64_t M, N, D;
        if (!inst[i].d_x || !inst[i].d_imfs) {
            plan->err = "null input or output pointer in the batch";
            return SEMD_EINVAL;
        }
        if (!geometry(plan->p, inst[i].rows, inst[i].cols, plan->p.order, M, N, D, plan->err))
            return SEMD_EINVAL;
        if (serial_length(M, N, D) > Lp) {
            plan->err = "an input is larger than the plan's shape";
            return SEMD_EBUDGET;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    return plan->p.precision == SEMD_FP64
               ? decompose_impl<double>(*plan, count, inst, nullptr, n_imfs, s, 0)
               : decompose_impl<float>(*plan, count, inst, nullptr, n_imfs, s, 0);
}

semd_status serial_emd_decompose_slices(semd_plan_t plan, const void *d_x, int64_t rows,
                                        int64_t cols, void *d_imfs, double *d_residue,
                                        int *n_imfs, void *stream)
{
    if (!plan)
        return SEMD_EINVAL;
    if (!d_x || !d_imfs) {
        plan->err = "null input or output pointer";
        return SEMD_EINVAL;
    }
    if (plan->p.ensemble_trials > 1) {
        plan->err = "slice-wise decomposition takes EMD plans only";
        return SEMD_EINVAL;
    }
    if (rows < 1 || cols < 1 || rows > plan->ws.cap_inst) {
        plan->err = "rows must be in [1, max_batch] and cols >= 1";
        return SEMD_EINVAL;
    }
    if (cols > plan->L) {
        plan->err = "a slice is longer than the plan's serialized length";
        return SEMD_EBUDGET;
    }
    // signal i = row i, decomposed alone (one row: no serialization, no transitions); IMF
    // k of signal i lands at k * rows * cols + i * cols
    const size_t elem = plan->p.precision == SEMD_FP64 ? 8 : 4;
    std::vector<semd_instance> in((size_t)rows);
    for (int64_t i = 0; i < rows; ++i)
        in[(size_t)i] = semd_instance{(const char *)d_x + (size_t)(i * cols) * elem, 1, cols,
                                      (char *)d_imfs + (size_t)(i * cols) * elem,
                                      d_residue ? d_residue + i * cols : nullptr};
    cudaStream_t s = (cudaStream_t)stream;
    const semd_params saved = plan->p;
    plan->p.order = SEMD_ORDER_ROWS;
    const semd_status st =
        plan->p.precision == SEMD_FP64
            ? decompose_impl<double>(*plan, (int)rows, in.data(), nullptr, n_imfs, s, rows * cols)
            : decompose_impl<float>(*plan, (int)rows, in.data(), nullptr, n_imfs, s, rows * cols);
    plan->p = saved;
    return st;
}

semd_status serial_emd_ceemdan(semd_plan_t plan, const void *d_x, const void *d_noise,
                               void *d_modes, double *d_residue, int *n_modes, void *stream)
{
    if (!plan)
        return SEMD_EINVAL;
    if (plan->p.ensemble_trials < 2) {
        plan->err = "CEEMDAN takes ensemble plans (ensemble_trials >= 2)";
        return SEMD_EINVAL;
    }
    if (!d_x || !d_noise || !d_modes) {
        plan->err = "null input, noise or output pointer";
        return SEMD_EINVAL;
    }
    if (plan->p.ensemble_trials > 65535) {
        plan->err = "CEEMDAN takes at most 65535 realizations";
        return SEMD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return plan->p.precision == SEMD_FP64
               ? ceemdan_impl<double>(*plan, d_x, d_noise, d_modes, d_residue, n_modes, s)
               : ceemdan_impl<float>(*plan, d_x, d_noise, d_modes, d_residue, n_modes, s);
}

semd_status serial_emd_plan_counts(semd_plan_t plan, int count, int *n_imfs, int *sifts)
{
    if (!plan || count < 0 || count > plan->last_count)
        return SEMD_EINVAL;
    plan->counts(count, n_imfs, sifts);
    return SEMD_OK;
}

semd_status serial_emd_extrema(semd_plan_t plan, const void *d_h, int64_t L, int32_t *d_tmax,
                               int32_t *d_tmin, int64_t *n_max, int64_t *n_min, void *stream)
{
    if (!plan || !d_h || !d_tmax || !d_tmin || !n_max || !n_min)
        return SEMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return plan->p.precision == SEMD_FP64
               ? extrema_impl<double>(*plan, d_h, L, d_tmax, d_tmin, n_max, n_min, s)
               : extrema_impl<float>(*plan, d_h, L, d_tmax, d_tmin, n_max, n_min, s);
}

semd_status serial_emd_sift(semd_plan_t plan, const void *d_h, int64_t L, void *d_out,
                            double *sd_num, double *sd_den, void *stream)
{
    if (!plan || !d_h || !d_out || !sd_num || !sd_den)
        return SEMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return plan->p.precision == SEMD_FP64
               ? sift_impl<double>(*plan, d_h, L, d_out, sd_num, sd_den, s)
               : sift_impl<float>(*plan, d_h, L, d_out, sd_num, sd_den, s);
}

void serial_emd_destroy(semd_plan_t plan)
{
    if (!plan)
        return;
    if (plan->gstream)
        cudaStreamSynchronize(plan->gstream);
    if (plan->graph_exec)
        cudaGraphExecDestroy(plan->graph_exec);
    if (plan->ce_graph_exec)
        cudaGraphExecDestroy(plan->ce_graph_exec);
    if (plan->ev_in)
        cudaEventDestroy(plan->ev_in);
    if (plan->ev_out)
        cudaEventDestroy(plan->ev_out);
    if (plan->gstream)
        cudaStreamDestroy(plan->gstream);
    if (plan->lstream)
        cudaStreamDestroy(plan->lstream);
    plan->prof.destroy();
    plan->ws.release();
    delete plan;
}

semd_status serial_emd_plan_set_tile(semd_plan_t plan, int tile)
{
    if (!plan)
        return SEMD_EINVAL;
    if (tile == 0) {
        int ctas, variant;
        choose_pass_shape(plan->p, plan->L, plan->ws.cap_inst, tile, ctas, variant);
    }
    if (tile != 128 && tile != 256 && tile != 512) {
        plan->err = "tile must be 0, 128, 256 or 512";
        return SEMD_EINVAL;
    }
    plan->ws.tile = tile;
    return SEMD_OK;
}

int serial_emd_plan_get_tile(semd_plan_t plan) { return plan ? plan->ws.tile : 0; }

semd_status serial_emd_plan_set_pass_ctas(semd_plan_t plan, int ctas_per_sm)
{
    if (!plan)
        return SEMD_EINVAL;
    if (ctas_per_sm < 0 || ctas_per_sm > 64) {
        plan->err = "ctas_per_sm must be in [0, 64]";
        return SEMD_EINVAL;
    }
    plan->ws.pass_ctas = ctas_per_sm;
    return SEMD_OK;
}

int serial_emd_plan_get_pass_ctas(semd_plan_t plan) { return plan ? plan->ws.pass_ctas : 0; }

semd_status serial_emd_plan_set_pass_variant(semd_plan_t plan, int variant)
{
    if (!plan)
        return SEMD_EINVAL;
    if (variant != 0 && variant != 1) {
        plan->err = "variant must be 0 or 1";
        return SEMD_EINVAL;
    }
    plan->ws.pass_variant = variant;
    return SEMD_OK;
}

int serial_emd_plan_get_pass_variant(semd_plan_t plan) { return plan ? plan->ws.pass_variant : 0; }

semd_status serial_emd_plan_set_options(semd_plan_t plan, int use_graphs, int profile)
{
    if (!plan)
        return SEMD_EINVAL;
    plan->graphs = use_graphs != 0;
    plan->prof.on = profile != 0;
    return SEMD_OK;
}

semd_status serial_emd_plan_stats(semd_plan_t plan, semd_stats *out)
{
    if (!plan || !out)
        return SEMD_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->kernel_launches = plan->stat_launches;
    out->used_graph = plan->stat_graph;
    out->sample_sifts = (int64_t)plan->ws.h_stats->sample_sifts;
    out->pass_bytes = (int64_t)plan->ws.h_stats->pass_bytes;
    double ms[2];
    int64_t cnt[2];
    plan->prof.totals(ms, cnt);
    out->pass_launches = cnt[0];
    out->pass_ms = ms[0];
    out->reduce_launches = cnt[1];
    out->reduce_ms = ms[1];
    return SEMD_OK;
}

semd_status serial_emd_eemd_trial(semd_plan_t plan, int trial, void *d_imfs, double *d_residue,
                                  int *n_imfs, double *beta, void *stream)
{
    if (!plan)
        return SEMD_EINVAL;
    if (plan->p.ensemble_trials < 2 || plan->last_ceemdan || plan->last_ninst < 2) {
        plan->err = "no EEMD decomposition has run on this plan";
        return SEMD_EINVAL;
    }
    if (trial < 0 || trial >= plan->last_ninst || !d_imfs) {
        plan->err = "trial out of range or null output";
        return SEMD_EINVAL;
    }
    std::string &err = plan->err;
    Workspace &ws = plan->ws;
    cudaStream_t s = (cudaStream_t)stream;
    const int K = plan->p.max_imfs;
    const unsigned grid = (unsigned)std::min<int64_t>((plan->L + 255) / 256, 4 * 152);
    if (plan->p.precision == SEMD_FP64)
        k_eemd_trial<double><<<grid, 256, 0, s>>>(ws.d_inst, ws.d_state, trial, K,
                                                  (const double *)ws.eemd_scratch,
                                                  (double *)d_imfs, d_residue);
    else
        k_eemd_trial<float><<<grid, 256, 0, s>>>(ws.d_inst, ws.d_state, trial, K,
                                                 (const float *)ws.eemd_scratch,
                                                 (float *)d_imfs, d_residue);
    SEMD_CU(cudaGetLastError());
    if (beta) {
        SEMD_CU(cudaMemcpyAsync(beta, ws.d_beta, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    if (beta || n_imfs)
        SEMD_CU(cudaStreamSynchronize(s));
    if (n_imfs)
        *n_imfs = ws.h_state[trial].imf_count;
    return SEMD_OK;
}

semd_status serial_emd_plan_set_noise_seed(semd_plan_t plan, uint64_t seed)
{
    if (!plan)
        return SEMD_EINVAL;
    plan->noise_seed = seed;
    return SEMD_OK;
}

semd_status serial_emd_interface_solve_shape(int precision, int spline_end, int *cluster,
                                             int64_t *min_tiles, int64_t *max_tiles)
{
    if (!cluster || !min_tiles || !max_tiles ||
        (precision != SEMD_FP64 && precision != SEMD_FP32_MIXED) ||
        (spline_end != SEMD_SPLINE_NATURAL && spline_end != SEMD_SPLINE_NOT_A_KNOT))
        return SEMD_EINVAL;
    const size_t elem = precision == SEMD_FP64 ? 8 : 4;
    if (setup_kernel_attrs(elem) != cudaSuccess) {
        cudaGetLastError();
        return SEMD_ECUDA;
    }
    ReduceArgs ra{};
    ra.spline_end = spline_end;
    set_reduce_shape(ra, 1, 1, elem);
    *cluster = ra.cl;
    *min_tiles = ra.cl_min_nt;
    *max_tiles = ra.cl_max_nt;
    return SEMD_OK;
}

int64_t serial_emd_plan_launch_times(semd_plan_t plan, int kind, float *ms, int64_t cap)
{
    if (!plan || (kind != 0 && kind != 1) || cap < 0)
        return -1;
    return plan->prof.times(kind, ms, cap);
}

const char *serial_emd_last_error(semd_plan_t plan)
{
    return plan ? plan->err.c_str() : g_plan_create_error.c_str();
}

} // extern "C"

// ================================================================= allocation-free sift
//
// serial_emd_sift_noalloc: the single sift of serial_emd_sift without a plan. Its
// scratch (signal and residue buffers, per-tile records of the spline solve, the
// instance descriptor and state) lives in one file-scope __device__ array, so a call
// reserves no device memory. Every GPU that loads this library holds the array
// (kNoAllocBytes, about 2.4 MB) until the process exits. All calls share it: calls
// that overlap on the GPU (concurrent streams, threads or devices sharing a context)
// race on it, and each call clears what it needs before use.
namespace semd {

constexpr int64_t kNoAllocMaxL = 65536;                  // largest accepted L
constexpr int kNoAllocTiles = (int)(kNoAllocMaxL / kTile);
constexpr int64_t kNoAllocRent = 2 * rscr_env_doubles(reduce_len(kNoAllocTiles)); // doubles
constexpr size_t na_round(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kNoAllocBytes =
    4 * na_round(kNoAllocMaxL * 8) +                        // h0, h1 (sized for FP64), r0, r1
    na_round(sizeof(Inst)) + na_round(sizeof(State)) + na_round(kNoAllocTiles * 4) +
    na_round(kNoAllocTiles * 2 * tile_rec_bytes(8)) +
    na_round(kNoAllocTiles * 2 * sizeof(TileSolve)) + na_round(kNoAllocTiles * sizeof(TileAux)) +
    na_round(kNoAllocTiles * 32 * sizeof(uint2)) +
    na_round(kNoAllocRent * 8) +
    na_round(8) + na_round(sizeof(Stats)) + na_round(4 * 8); // active flags, stats, result

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_base[kNoAllocMaxDevices];

// Once per device, with that device current: the device address of the scratch array
// (its host-side name is only a stand-in) and the shared-memory limits of the kernels.
static semd_status noalloc_setup(void *&base, std::string &err)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return SEMD_ECUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        err = "device ordinal out of range for the allocation-free sift";
        return SEMD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress of the static scratch: ") +
                  cudaGetErrorString(e);
            return SEMD_ECUDA;
        }
        e = set_smem_attr<float>();
        if (e == cudaSuccess)
            e = set_smem_attr<double>();
        if (e != cudaSuccess) {
            err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
            return SEMD_ECUDA;
        }
        g_noalloc_base[dev] = p;
    }
    base = g_noalloc_base[dev];
    return SEMD_OK;
}

// Clears the per-call state and writes the instance descriptor (passed by value, so
// no host staging buffer is needed).
__global__ void k_noalloc_setup(Inst in, Inst *d_inst, State *d_state, int32_t *tile_inst,
                                int ntiles, int32_t *active, Stats *stats)
{
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        tile_inst[t] = 0;
    if (threadIdx.x == 0) {
        *d_inst = in;
        *d_state = State{};
        active[0] = 0;
        active[1] = 0;
        *stats = Stats{};
    }
}

// The sums (h - h')^2 and h^2 over the tiles, in tile order, and the state's mode.
__global__ void k_noalloc_result(const State *st, const TileAux *taux, int ntiles, double *out)
{
    if (threadIdx.x != 0)
        return;
    double a = 0.0, b = 0.0;
    for (int t = 0; t < ntiles; ++t) {
        a += taux[t].sd_num;
        b += taux[t].sd_den;
    }
    out[0] = a;
    out[1] = b;
    out[2] = (double)st->mode;
}

template <typename R>
static semd_status sift_noalloc_impl(const semd_params &p, const void *d_h, int64_t L,
                                     void *d_out, double *sd_num, double *sd_den,
                                     cudaStream_t s, std::string &err)
{
    void *base = nullptr;
    semd_status st = noalloc_setup(base, err);
    if (st != SEMD_OK)
        return st;
    const int ntiles = (int)((L + kTile - 1) / kTile);
    Workspace ws; // views into the static scratch; never allocated or released
    char *cur = (char *)base;
    auto take = [&cur](size_t bytes) {
        void *q = cur;
        cur += na_round(bytes);
        return q;
    };
    ws.h0 = take(kNoAllocMaxL * 8);
    ws.h1 = take(kNoAllocMaxL * 8);
    ws.r0 = (double *)take(kNoAllocMaxL * 8);
    ws.r1 = (double *)take(kNoAllocMaxL * 8);
    ws.d_inst = (Inst *)take(sizeof(Inst));
    ws.d_state = (State *)take(sizeof(State));
    ws.d_tile_inst = (int32_t *)take(kNoAllocTiles * 4);
    ws.d_tex = take(kNoAllocTiles * 2 * tile_rec_bytes(8));
    ws.d_tsol = (TileSolve *)take(kNoAllocTiles * 2 * sizeof(TileSolve));
    ws.d_taux = (TileAux *)take(kNoAllocTiles * sizeof(TileAux));
    ws.d_kmask = (uint2 *)take(kNoAllocTiles * 32 * sizeof(uint2));
    ws.d_rscr = (double *)take(kNoAllocRent * 8);
    ws.d_active = (int32_t *)take(8);
    ws.d_stats = (Stats *)take(sizeof(Stats));
    double *d_result = (double *)take(4 * 8);
    ws.max_ntiles = ntiles;
    ws.min_ntiles = ntiles;
    ws.tile = kTile;
    ws.elem_size = sizeof(R);

    Inst in{};
    in.L = L;
    in.M = L;
    in.N = 1;
    in.D = 0;
    bind_instance(ws, in, 0, 0, 0);
    k_noalloc_setup<<<1, 64, 0, s>>>(in, ws.d_inst, ws.d_state, ws.d_tile_inst, ntiles,
                                     ws.d_active, ws.d_stats);
    k_to_double<R><<<152, 256, 0, s>>>((const R *)d_h, L, ws.r0);
    semd_params q = p;
    q.stop = SEMD_STOP_FIXED;
    q.fixed_sifts = 1000; // stay in SIFT mode
    q.max_imfs = 1;
    ReduceArgs ra = reduce_args(ws, q);
    launch_pass<R>(ws, ntiles, true, false, s); // INIT: h = r, export
    launch_reduce<R>(ra, 1, s);
    launch_pass<R>(ws, ntiles, true, false, s); // SIFT
    k_noalloc_result<<<1, 32, 0, s>>>(ws.d_state, ws.d_taux, ntiles, d_result);
    SEMD_CU(cudaGetLastError());
    double res[3];
    SEMD_CU(cudaMemcpyAsync(res, d_result, sizeof(res), cudaMemcpyDeviceToHost, s));
    SEMD_CU(cudaStreamSynchronize(s));
    if ((int)res[2] != MODE_SIFT) {
        err = "the signal lacks maxima or minima; it cannot be sifted";
        return SEMD_EINVAL;
    }
    // the SIFT pass read h from buffer hpar = 1 and wrote buffer 0
    SEMD_CU(cudaMemcpyAsync(d_out, ws.h0, (size_t)L * sizeof(R), cudaMemcpyDeviceToDevice, s));
    *sd_num = res[0];
    *sd_den = res[1];
    return SEMD_OK;
}

} // namespace semd

extern "C" semd_status serial_emd_sift_noalloc(const semd_params *params, const void *d_h,
                                               int64_t L, void *d_out, double *sd_num,
                                               double *sd_den, void *stream)
{
    std::string &err = semd::g_plan_create_error;
    err.clear();
    if (!params || !d_h || !d_out || !sd_num || !sd_den) {
        err = "null argument";
        return SEMD_EINVAL;
    }
    if (params->precision != SEMD_FP64 && params->precision != SEMD_FP32_MIXED)
        return err = "precision must be FP64 or FP32_MIXED", SEMD_EINVAL;
    if (params->boundary != SEMD_BOUNDARY_MIRROR && params->boundary != SEMD_BOUNDARY_ENDPOINTS)
        return err = "boundary must be MIRROR or ENDPOINTS", SEMD_EINVAL;
    if (params->boundary == SEMD_BOUNDARY_MIRROR &&
        (params->mirror_knots < 1 || params->mirror_knots > 2))
        return err = "mirror_knots must be 1 or 2", SEMD_EINVAL;
    if (params->spline_end != SEMD_SPLINE_NATURAL && params->spline_end != SEMD_SPLINE_NOT_A_KNOT)
        return err = "spline_end must be NATURAL or NOT_A_KNOT", SEMD_EINVAL;
    if (L < 1 || L > semd::kNoAllocMaxL) {
        err = "L = " + std::to_string(L) + " is outside [1, " +
              std::to_string(semd::kNoAllocMaxL) + "], the size of the allocation-free scratch";
        return SEMD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return params->precision == SEMD_FP64
               ? semd::sift_noalloc_impl<double>(*params, d_h, L, d_out, sd_num, sd_den, s, err)
               : semd::sift_noalloc_impl<float>(*params, d_h, L, d_out, sd_num, sd_den, s, err);
}
