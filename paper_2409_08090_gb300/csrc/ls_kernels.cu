// Kernels of the single-series Lomb-Scargle NUFFT pipeline (arXiv 2409.08090,
// Sec. 1): FP64 preprocessing, bin sort, pass A (spread + column FFTs) and
// pass B (row FFTs + deconvolution + power).
//
// Notation.  Frequencies f_k = f0 + k df, k < nf; K0 = floor(nf/2), centre
// fc = f0 + K0 df, centred mode k' = k - K0.  For a point at time t:
//   x  = 2 pi frac(df t)          (NUFFT coordinate for the f transforms)
//   2x = 2 pi frac(2 df t)        (coordinate for the 2f transform)
//   p  = exp(2 pi i frac(fc t))   (pre-phase that centres the modes)
// so that sum_j h_j exp(2 pi i f_k t_j) = sum_j (h_j p_j) exp(i k' x_j) and
// sum_j h_j exp(4 pi i f_k t_j) = sum_j (h_j p_j^2) exp(i k' 2x_j): three type-1
// transforms (Eq. 2) with strengths s1 = w^ y' p, s2 = w^ p (coordinate x) and
// s3 = w^ p^2 (coordinate 2x) over the same modes k'.
//
// Fine grid: n cells, cell m at 2 pi m / n.  Spreading uses the ES kernel
// psi(z) = exp(beta (sqrt(1 - z^2) - 1)) with z = (m - u) * 2 / w, u = x n / 2 pi.
// The FFT is four-step: m = a + N1 b; pass A transforms each column a over b
// (length N2) and applies exp(2 pi i a d / n); pass B transforms each row d over
// a (length N1) giving mode k = d + N2 c, k' = k or k - n.
#include <atomic>
#include <math.h>
#include <string.h>

#include <cooperative_groups.h>

#include <mutex>
#include <utility>
#include <vector>

#include "ls_fft.cuh"
#include "ls_internal.cuh"

namespace nls {

template <typename T> using Cplx = typename Cx<T>::type;

__device__ __forceinline__ SeriesDesc series_of(const Batch &b, int s)
{
    return b.many ? b.many[s] : b.one;
}

template <typename T>
__device__ __forceinline__ PointSet<T> shifted(PointSet<T> p, int64_t off)
{
    p.ab += off;
    p.roff += off;
    p.s[0] += off;
    p.s[1] += off;
    p.rank += off;
    return p;
}

// ---------------------------------------------------------------------------
// Block reduction helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block (blockDim.x multiple of 32, <= 1024); result valid
// in thread 0.  Fixed order, hence deterministic.
__device__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Returns true in every thread of the block that finished last (all partials
// of the grid are then visible).
__device__ bool last_block(unsigned int *counter)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    return is_last;
}

// Finite-value and positivity tests on the bit pattern (integer pipe).
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) !=
           0x7ff0000000000000ull;
}

// 1/x in FP64 from an FP32 reciprocal and one Newton step (relative error
// below 4e-15; the FP64 divide is a long sequence on a part whose FP64 rate is
// 1/64 of FP32).  The exponent test on the bits keeps x within FP32 range;
// otherwise the divide is used.
__device__ __forceinline__ double rcp_fp64(double x)
{
    const int ex = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
    if (ex < 1023 - 120 || ex > 1023 + 120) return 1.0 / x;
    const double r = (double)__frcp_rn((float)x);
    return fma(r, fma(-x, r, 1.0), r);
}

// Sum of `width` interleaved partial sums over `nparts` blocks, by the whole
// (last) block in a fixed order; results valid in thread 0.
__device__ void reduce_partials(const double *partials, int nparts, int width, double *out,
                                double *sh)
{
    for (int c = 0; c < width; ++c) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += __ldcg(partials + width * i + c);
        out[c] = block_sum(v, sh);
    }
}

// ---------------------------------------------------------------------------
// K1a: weights and weighted mean (FP64).  w_j = 1/dy_j^2 (kept for k_points),
// W = sum w_j, WY = sum w_j y_j, WY2 = sum w_j y_j^2.  The one-pass variance
// WY2/W - ybar^2 only sets the scale of the strengths (the power does not
// depend on it); the exact YY comes from the second pass.  Without centring (center = 0) ybar is taken as
// 0 and the scale follows the mean square.
// ---------------------------------------------------------------------------
__global__ void k_stats(const double *__restrict__ t, const double *__restrict__ y,
                        const double *__restrict__ dy, Batch bt, double *partials,
                        unsigned int *counter, Stats *st, int *status, int center, double *wts)
{
    const int ser = blockIdx.y;
    const SeriesDesc sd = series_of(bt, ser);
    t += sd.pt_off;
    y += sd.y_off;
    if (dy) dy += sd.pt_off;
    const int64_t nd = sd.nd;
    const int64_t nch = (nd + kRedChunk - 1) / kRedChunk;
    wts += sd.rec_off;                    // w_j at the series' records, for k_points
    partials += 3 * red_row0(sd.rec_off, ser);
    counter += 2 * ser;
    st += ser;
    __shared__ double sh[32];
    bool ok = true;
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        double sw = 0.0, swy = 0.0, swy2 = 0.0;
        const int64_t j1 = min(nd, (c + 1) * kRedChunk);
        for (int64_t j = c * kRedChunk + threadIdx.x; j < j1; j += blockDim.x) {
            const double d = dy ? dy[j] : 1.0;
            const double yj = y[j];
            ok &= finite_bits(d) && finite_bits(yj) && finite_bits(t[j]) &&
                  __double_as_longlong(d) > 0;
            const double w = rcp_fp64(d * d);
            wts[j] = w;
            const double wy = w * yj;
            sw += w;
            swy += wy;
            swy2 = fma(wy, yj, swy2);
        }
        const double a = block_sum(sw, sh);
        const double b = block_sum(swy, sh);
        const double q = block_sum(swy2, sh);
        if (threadIdx.x == 0) {
            partials[3 * c] = a;
            partials[3 * c + 1] = b;
            partials[3 * c + 2] = q;
        }
    }
    if (!ok) atomicOr(status, kStatBadInput);
    if (last_block(counter)) {
        double r[3];
        reduce_partials(partials, (int)nch, 3, r, sh);
        if (threadIdx.x == 0) {
            const double W = r[0], WY = r[1], WY2 = r[2];
            st->W = W;
            st->WY = WY;
            st->WY2 = WY2;
            st->ybar = center ? WY / W : 0.0;
            st->invW = 1.0 / W;
            const double m2 = WY2 / W;
            const double var = fmax(m2 - st->ybar * st->ybar, 1e-20 * m2);
            st->scale = (var > 0.0 && isfinite(var)) ? 1.0 / sqrt(var) : 1.0;
            st->smax[0] = st->smax[1] = st->smax[2] = 0u;   // k_points takes the maxima
            *counter = 0u;
        }
    }
}

// The pass-B scalars of a series, once YY (scaled) is known.
__device__ __forceinline__ void finish_series_stats(Stats *st)
{
    const double YY = st->YY;
    st->psd = 0.5 * st->W * YY / (st->scale * st->scale);
    st->unscale = 1.0 / st->scale;
    st->yy_hi = (float)YY;
    st->yy_lo = (float)(YY - (double)st->yy_hi);
}

// ---------------------------------------------------------------------------
// Exact phase reduction in integer arithmetic.  A double f = +-m 2^e (m < 2^53)
// times a double t is the 106-bit integer product of the mantissas times a
// power of two, so frac(f t) is a bit field of that product: it is taken as a
// 128-bit fixed-point fraction (value F / 2^128), exact up to truncation below
// 2^-128, on the integer pipe.  frac((f0 + K0 df) t) = frac(frac(f0 t) +
// K0 frac(df t)) then follows by 128-bit modular arithmetic.
// ---------------------------------------------------------------------------
typedef unsigned __int128 u128;

__device__ __forceinline__ u128 frac_fixed(uint64_t fm, int fe, int fneg, double t)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    const int ex = (int)((b >> 52) & 0x7ff);
    const uint64_t tm = (b & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull);
    const int sh = fe + (ex ? ex : 1) - 1075 + 128;   // F = P 2^sh mod 2^128
    const u128 P = (u128)fm * tm;
    u128 F;
    if (sh >= 128) F = 0;
    else if (sh >= 0) F = P << sh;
    else if (sh > -128) F = P >> (-sh);
    else F = 0;
    return (fneg ^ (int)(b >> 63)) ? (u128)0 - F : F;
}

// Cell split of the coordinate frac * n: c0 = ceil(u - w/2) packed as
// a | (b << 16) with c0 = a + N1 b, and roff = c0 - u + w/2 in [0, 1], from
// the 128-bit fraction (u = F n / 2^128 to within n 2^-128 cells).
template <typename T>
__device__ __forceinline__ void split_fixed(u128 F, const Geometry &g, uint32_t &ab, T &roff)
{
    const u128 U = (u128)(uint64_t)(F >> 64) * (uint64_t)g.n +
                   (((u128)(uint64_t)F * (uint64_t)g.n) >> 64);
    const int ui = (int)(uint64_t)(U >> 64);       // floor(u)
    const uint64_t uf = (uint64_t)U;               // frac(u) 2^64
    int c0;
    u128 R;                                        // roff 2^64
    if (g.w & 1) {
        const bool up = uf > 0x8000000000000000ull;
        c0 = ui - (g.w - 1) / 2 + (up ? 1 : 0);
        R = ((u128)(up ? 3u : 1u) << 63) - uf;
    } else {
        const bool up = uf != 0;
        c0 = ui - g.w / 2 + (up ? 1 : 0);
        R = ((u128)(up ? 1u : 0u) << 64) - uf;
    }
    if (c0 < 0) c0 += (int)g.n;
    if (c0 >= (int)g.n) c0 -= (int)g.n;
    const int bb = c0 / g.N1;
    ab = (uint32_t)(c0 - bb * g.N1) | ((uint32_t)bb << 16);
    if (sizeof(T) == 4) roff = (T)((float)(uint32_t)(uint64_t)(R >> 40) * 0x1p-24f);   // R <= 2^64
    else roff = (T)((double)(uint64_t)(R >> 11) * 0x1p-53);
}

// exp(2 pi i phase) for a fixed-point phase.
template <typename T> struct Cis;

template <> struct Cis<double> {
    __device__ __forceinline__ static double2 of(u128 F) {
        const double c = (double)(long long)(uint64_t)(F >> 64) * 0x1p-64;   // in [-1/2, 1/2)
        double s, co;
        sincospi(2.0 * c, &s, &co);
        return make_double2(co, s);
    }
};

// FP32 path: the phase c = s 2^-64 (in cycles, [-1/2, 1/2)) is split as
// cf + dc with cf = floor(c 2^24) 2^-24 (exact in FP32) and dc the remainder
// (in radians, 0 <= dc < 2 pi 2^-24, its 32 leading bits converted);
// sincospif(2 cf) is corrected to first order in dc (neglected term
// dc^2 / 2 < 7e-14).  Only 32-bit conversions: this part converts 64-bit
// integers at its FP64 rate.
template <> struct Cis<float> {
    __device__ __forceinline__ static float2 of(u128 F) {
        const long long s = (long long)(uint64_t)(F >> 64);
        const int hi = (int)(s >> 40);                                         // |hi| <= 2^23
        const unsigned rem = (unsigned)(((unsigned long long)s & 0xFFFFFFFFFFull) >> 8);
        const float cf = (float)hi * 0x1p-24f;
        const float dc = 6.2831853071795865f * ((float)rem * 0x1p-56f);
        float sn, co;
        sincospif(2.0f * cf, &sn, &co);
        return make_float2(fmaf(-dc, sn, co), fmaf(dc, co, sn));
    }
};

// Stable rank of this lane's key among the warp's earlier keys, continuing
// the warp-private counts cnt[key] (which it then advances): lanes with equal
// keys (peers: this lane's match mask among the active lanes) are ranked in lane
// order after everything counted before.  Inactive lanes take no part; the
// result is 0 for them.  Warp-uniform call.
__device__ __forceinline__ int warp_stable_rank(unsigned short *cnt, int key, bool active,
                                                unsigned peers)
{
    const unsigned lane = threadIdx.x & 31u;
    int base = 0, r = 0;
    if (active) {
        base = cnt[key];
        r = base + __popc(peers & ((1u << lane) - 1u));
    }
    __syncwarp();
    if (active && (int)lane == __ffs(peers) - 1) cnt[key] = (unsigned short)(base + __popc(peers));
    __syncwarp();
    return r;
}

// Bits of an FP32 upper bound of max(|s.x|, |s.y|) (ordered like the value).
__device__ __forceinline__ unsigned strength_bound_bits(float2 s)
{
    return __float_as_uint(fmaxf(fabsf(s.x), fabsf(s.y)));
}
__device__ __forceinline__ unsigned strength_bound_bits(double2 s)
{
    return __float_as_uint(__double2float_ru(fmax(fabs(s.x), fabs(s.y))));
}


// ---------------------------------------------------------------------------
// K1b: per-point records + YY reduction.  Coordinates and pre-phases come
// from the exact integer reduction; weights and the mean-subtracted data are
// FP64; strengths are stored in T.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_points(const double *__restrict__ t, const double *__restrict__ y,
                         const double *__restrict__ wts, Batch bt, Geometry g, PointSet<T> px,
                         PointSet<T> p2, double *partials, unsigned int *counter, Stats *st,
                         int *status)
{
    const int ser = blockIdx.y;
    const SeriesDesc sd = series_of(bt, ser);
    t += sd.pt_off;
    y += sd.y_off;
    wts += sd.rec_off;                    // w_j = 1/dy_j^2 from k_stats
    const int64_t nd = sd.nd;
    const PhaseArgs ph = sd.ph;
    px = shifted(px, sd.rec_off);
    p2 = shifted(p2, sd.rec_off);
    const int64_t nch = (nd + kRedChunk - 1) / kRedChunk;
    partials += 3 * red_row0(sd.rec_off, ser);
    counter += 2 * ser + 1;
    st += ser;
    __shared__ double sh[32];
    const double invW = st->invW;
    const double ybar = st->ybar;
    const double scale = st->scale;
    unsigned m1 = 0u, m2 = 0u, m3 = 0u;   // strength bounds (bits), this thread's records
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        double syy = 0.0, sy2 = 0.0;
        const int64_t j1 = min(nd, (c + 1) * kRedChunk);
        for (int64_t j = c * kRedChunk + threadIdx.x; j < j1; j += blockDim.x) {
            const double tj = t[j], yj = y[j];
            const double wh = wts[j] * invW;
            const double yc = yj - ybar;
            const double wyc = wh * yc;
            syy = fma(wyc, yc, syy);
            sy2 = fma(wh * yj, yj, sy2);
            const u128 Fx = frac_fixed(ph.df_m, ph.df_e, 0, tj);          // frac(df t)
            const u128 Fc = frac_fixed(ph.f0_m, ph.f0_e, ph.f0_neg, tj)
                          + (u128)(uint64_t)ph.K0 * Fx;                   // frac(fc t)
            uint32_t ab1, ab2;
            T r1, r2;
            split_fixed<T>(Fx, g, ab1, r1);
            split_fixed<T>(Fx << 1, g, ab2, r2);
            const Cplx<T> p = Cis<T>::of(Fc);
            const Cplx<T> q = Cis<T>::of(Fc << 1);
            const T at = (T)(wyc * scale), wt = (T)wh;
            const Cplx<T> s1 = mk2(at * p.x, at * p.y), s2 = mk2(wt * p.x, wt * p.y),
                          s3 = mk2(wt * q.x, wt * q.y);
            px.ab[j] = ab1;
            px.roff[j] = r1;
            px.s[0][j] = s1;
            px.s[1][j] = s2;
            p2.ab[j] = ab2;
            p2.roff[j] = r2;
            p2.s[0][j] = s3;
            m1 = max(m1, strength_bound_bits(s1));
            m2 = max(m2, strength_bound_bits(s2));
            m3 = max(m3, strength_bound_bits(s3));
        }
        const double a = block_sum(syy, sh);
        const double b = block_sum(sy2, sh);
        if (threadIdx.x == 0) {
            partials[2 * c] = a;
            partials[2 * c + 1] = b;
        }
    }
    {
        m1 = __reduce_max_sync(0xffffffffu, m1);
        m2 = __reduce_max_sync(0xffffffffu, m2);
        m3 = __reduce_max_sync(0xffffffffu, m3);
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&st->smax[0], m1);
            atomicMax(&st->smax[1], m2);
            atomicMax(&st->smax[2], m3);
        }
    }
    if (last_block(counter)) {
        double r[2];
        reduce_partials(partials, (int)nch, 2, r, sh);
        if (threadIdx.x == 0) {
            const double YY = r[0], Y2 = r[1];
            st->YY = YY * st->scale * st->scale;
            st->Y2 = Y2;
            finish_series_stats(st);
            // A constant series: variance zero up to the rounding of the mean.
            if (!(YY > 1e-24 * Y2)) atomicOr(status, kStatDegenerate);
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// K1c: stable in-chunk bin ranks and the chunk histograms.  A block takes
// chunks of kChunk consecutive records (warp w the records w kChunk/8 .. of
// the chunk, 32 at a time), ranks every record among the chunk's earlier
// records of its bin (warp-private counts, then an exclusive scan over the
// warps) and writes the chunk's bin counts to its row of chist.  Dynamic
// shared memory: 2 x 8 x nbins 16-bit counts.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreadsPts)
k_rank(Batch bt, Geometry g, const uint32_t *__restrict__ abx, const uint32_t *__restrict__ ab2x,
       uint32_t *rank, int *chist)
{
    extern __shared__ __align__(16) unsigned short wcnt[];   // [geometry][warp][bin]
    constexpr int kWarps = kThreadsPts / 32;
    constexpr int kSteps = kChunk / kThreadsPts;             // records per thread per chunk
    const int ser = blockIdx.y;
    const SeriesDesc sd = series_of(bt, ser);
    const int64_t nd = sd.nd;
    abx += sd.rec_off;
    ab2x += sd.rec_off;
    rank += sd.rec_off;
    const int nbins = g.nbins;
    const int64_t row0 = chunk_row0(sd.rec_off, ser);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned short *cx = wcnt + (size_t)warp * nbins;                 // geometry x
    unsigned short *c2 = wcnt + (size_t)(kWarps + warp) * nbins;      // geometry 2x
    const int64_t nchunk = (nd + kChunk - 1) / kChunk;
    for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        __syncthreads();                      // the previous chunk is done with the counts
        for (int i = threadIdx.x; i < kWarps * nbins; i += blockDim.x)
            reinterpret_cast<uint32_t *>(wcnt)[i] = 0u;   // 2 x 8 x nbins 16-bit counts
        __syncthreads();
        uint32_t rk[kSteps], bins[kSteps];
        uint32_t a1[kSteps], a2[kSteps];
        const int64_t jw = ch * kChunk + (int64_t)warp * (kChunk / kWarps) + lane;
#pragma unroll
        for (int step = 0; step < kSteps; ++step) {      // all loads in flight first
            const int64_t j = jw + step * 32;
            a1[step] = j < nd ? __ldg(abx + j) : 0u;
            a2[step] = j < nd ? __ldg(ab2x + j) : 0u;
        }
#pragma unroll
        for (int step = 0; step < kSteps; ++step) {
            const bool act = jw + step * 32 < nd;
            const int b1 = (int)((a1[step] & 0xFFFFu) >> g.logBA);
            const int b2 = (int)((a2[step] & 0xFFFFu) >> g.logBA);
            bins[step] = (uint32_t)b1 | ((uint32_t)b2 << 16);
            const unsigned amask = __ballot_sync(0xffffffffu, act);
            const unsigned pe1 = __match_any_sync(0xffffffffu, act ? b1 : -1 - lane) & amask;
            const unsigned pe2 = __match_any_sync(0xffffffffu, act ? b2 : -1 - lane) & amask;
            rk[step] = (uint32_t)warp_stable_rank(cx, b1, act, pe1) |
                       ((uint32_t)warp_stable_rank(c2, b2, act, pe2) << 16);
        }
        __syncthreads();
        // exclusive scan of each bin's counts over the warps (input order), the
        // chunk's totals to its histogram row
        for (int col = threadIdx.x; col < 2 * nbins; col += blockDim.x) {
            const int geo = col >= nbins ? 1 : 0;
            unsigned short *c = wcnt + (size_t)geo * kWarps * nbins + (col - geo * nbins);
            int acc = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const int v = c[(size_t)w * nbins];
                c[(size_t)w * nbins] = (unsigned short)acc;
                acc += v;
            }
            chist[(row0 + ch) * 2 * nbins + col] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int step = 0; step < kSteps; ++step) {
            const int64_t j = jw + step * 32;
            if (j < nd) {
                const int b1 = (int)(bins[step] & 0xFFFFu), b2 = (int)(bins[step] >> 16);
                rank[j] = ((rk[step] & 0xFFFFu) + cx[b1]) | (((rk[step] >> 16) + c2[b2]) << 16);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K2a: per (geometry, bin) column of a series' chunk histograms: exclusive
// prefix over the chunks in place, and the column total to hist.  A block
// takes 32 columns (one per lane); warp w the rows w R .. (w + 1) R - 1,
// R = ceil(chunks / 8): each warp sums its rows, the warps' sums are scanned
// in shared memory, then each warp writes its rows' prefixes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_chunk_scan(Batch bt, int nbins, int *chist, int *hist)
{
    const int ser = blockIdx.y;
    const SeriesDesc sd = series_of(bt, ser);
    const int64_t nchunk = (sd.nd + kChunk - 1) / kChunk;
    const int ncol = 2 * nbins;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    __shared__ int part[8][32];
    const int64_t per = (nchunk + 7) / 8;
    const int64_t r0 = warp * per, r1 = min(nchunk, r0 + per);
    int *cp = chist + chunk_row0(sd.rec_off, ser) * ncol + col;
    int sum = 0;
    if (col < ncol) {
#pragma unroll 8
        for (int64_t r = r0; r < r1; ++r) sum += cp[r * ncol];
    }
    part[warp][lane] = sum;
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += part[w][lane];
    if (col < ncol) {
        for (int64_t r = r0; r < r1; ++r) {
            const int v = cp[r * ncol];
            cp[r * ncol] = off;
            off += v;
        }
        if (warp == 7) hist[(size_t)ser * ncol + col] = off;   // the column total
    }
}

// ---------------------------------------------------------------------------
// K2b: exclusive scan of the two bin-total arrays (one block per series) ->
// bin starts.
// ---------------------------------------------------------------------------
__global__ void k_scan(const int *__restrict__ hist, int nbins, int *binstart)
{
    hist += (size_t)blockIdx.x * 2 * nbins;
    binstart += (size_t)blockIdx.x * 2 * (nbins + 1);
    __shared__ int chunk_tot[1024];
    for (int geo = 0; geo < 2; ++geo) {
        const int *h = hist + geo * nbins;
        int *bs = binstart + geo * (nbins + 1);
        const int per = (nbins + blockDim.x - 1) / blockDim.x;
        const int lo = threadIdx.x * per;
        const int hi = min(nbins, lo + per);
        int s = 0;
        for (int i = lo; i < hi; ++i) s += h[i];
        chunk_tot[threadIdx.x] = s;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            int v = (threadIdx.x >= (unsigned)off) ? chunk_tot[threadIdx.x - off] : 0;
            __syncthreads();
            chunk_tot[threadIdx.x] += v;
            __syncthreads();
        }
        int run = (threadIdx.x == 0) ? 0 : chunk_tot[threadIdx.x - 1];
        for (int i = lo; i < hi; ++i) {
            bs[i] = run;
            run += h[i];
        }
        if (threadIdx.x == blockDim.x - 1) bs[nbins] = chunk_tot[blockDim.x - 1];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K2c: scatter the point records into bin order, stably: record j of chunk c
// goes to binstart[bin] + (records of its bin in chunks before c) + (its rank
// in chunk c), so a bin keeps its records in input order.  No atomics.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_scatter(Batch bt, Geometry g, PointSet<T> rx, PointSet<T> r2,
                          PointSet<T> sx, PointSet<T> s2, const int *__restrict__ binstart,
                          const int *__restrict__ chist, int *perm)
{
    const int ser = blockIdx.y;
    const SeriesDesc sd = series_of(bt, ser);
    const int64_t nd = sd.nd;
    rx = shifted(rx, sd.rec_off);
    r2 = shifted(r2, sd.rec_off);
    sx = shifted(sx, sd.rec_off);
    s2 = shifted(s2, sd.rec_off);
    const int nbins = g.nbins;
    const int *bs1 = binstart + (size_t)ser * 2 * (nbins + 1);
    const int *bs2 = bs1 + nbins + 1;
    const int *crow = chist + chunk_row0(sd.rec_off, ser) * 2 * nbins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nd; j += stride) {
        const uint32_t c1 = rx.ab[j], c2 = r2.ab[j], rk = rx.rank[j];
        const int b1 = (int)((c1 & 0xFFFFu) >> g.logBA), b2 = (int)((c2 & 0xFFFFu) >> g.logBA);
        const int *cr = crow + (j / kChunk) * 2 * nbins;
        const int d1 = __ldg(bs1 + b1) + __ldg(cr + b1) + (int)(rk & 0xFFFFu);
        const int d2 = __ldg(bs2 + b2) + __ldg(cr + nbins + b2) + (int)(rk >> 16);
        sx.ab[d1] = c1;
        sx.roff[d1] = rx.roff[j];
        sx.s[0][d1] = rx.s[0][j];
        sx.s[1][d1] = rx.s[1][j];
        s2.ab[d2] = c2;
        s2.roff[d2] = r2.roff[j];
        s2.s[0][d2] = r2.s[0][j];
        if (perm) perm[d1] = (int)j;      // shared-times batches: sorted -> input index
    }
}

// Integer division and remainder of non-negative 64-bit values by 32-bit
// divisors through the 32-bit unit when the operands fit (a 64-bit division
// is a long instruction sequence; these run in every thread of a block).
__device__ __forceinline__ int div_u32(int64_t num, int den)
{
    return num < 0x100000000ll ? (int)((uint32_t)num / (uint32_t)den) : (int)(num / den);
}
__device__ __forceinline__ int64_t mod_u32(int64_t p, int64_t n)
{
    return (p < 0x100000000ll && n < 0x100000000ll) ? (int64_t)((uint32_t)p % (uint32_t)n) : p % n;
}

// exp(2 pi i p / n) from the two-level four-step table, p in [0, n).
template <typename V>
__device__ __forceinline__ V tw4_root(const V *__restrict__ tw4, int64_t p)
{
    return cmul(__ldg(tw4 + (p & ((1 << kTw4Bits) - 1))),
                __ldg(tw4 + (1 << kTw4Bits) + (p >> kTw4Bits)));
}

// ---------------------------------------------------------------------------
// Fixed-point spreading.  Every cell of a column block is a sum of at most
// `count` contributions s_j psi (count = the block's records, psi <= 1), each
// at most maxs (the largest strength component among the block's bins) in
// magnitude, so |cell| <= maxs count <= 2^e.  Each contribution is rounded to
// a multiple of 2^(e - kBits) and the multiples are added exactly in integers
// (range 2^(kBits + 1): one bit of headroom for the rounding, whose total is at
// most count / 2 units).  Integer addition is associative, so a cell's value is
// the same whatever the order of its additions: every kernel and grouping of
// the spread gives bit-identical grids.  The rounding error per contribution is
// at most 2^(e - kBits - 1): with kBits = 30 (FP32 path) about 1e-9 of the
// block's bound, far below the FP32 tolerance, and with kBits = 62 (FP64 path)
// about 2e-19 of it.
// ---------------------------------------------------------------------------
template <typename T> struct Fixed;
template <> struct Fixed<float> {
    using I = int;
    static constexpr int kBits = 30;
    __device__ static int of(float x) { return __float2int_rn(x); }
    __device__ static void add(int *a, int v) { atomicAdd(a, v); }
};
template <> struct Fixed<double> {
    using I = long long;
    static constexpr int kBits = 62;
    __device__ static long long of(double x) { return __double2ll_rn(x); }
    __device__ static void add(long long *a, long long v)
    {
        atomicAdd(reinterpret_cast<unsigned long long *>(a), (unsigned long long)v);
    }
};

// x 2^k for a float x, by the exponent bits where 2^k is a normal float.
__device__ __forceinline__ float scale_pow2(float x, int k)
{
    return (k >= -126 && k <= 127) ? x * __int_as_float((k + 127) << 23) : ldexpf(x, k);
}

// The FP64 grid's cell v 2^(e - 62) as a double-float, on the integer and FP32
// pipes (this part converts and multiplies FP64 at 1/64 of the FP32 rate): the
// leading 24 bits of |v| and the next 24, rounded to nearest on the bit below
// them, as two exactly scaled floats, renormalised.  Relative error below 2^-48,
// the double-float's own precision.
__device__ __forceinline__ dfl fixed_to_dfl(long long v, int e)
{
    if (v == 0) return dfl(0.0f, 0.0f);
    const unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)m);
    const unsigned long long mn = m << lz;                   // leading bit at 63
    const unsigned h = (unsigned)(mn >> 40);                 // [2^23, 2^24)
    const unsigned l = (unsigned)((mn >> 16) & 0xFFFFFFull) + (unsigned)((mn >> 15) & 1ull);
    float hi = scale_pow2((float)h, e - 22 - lz);            // h 2^40 2^(e - 62 - lz)
    float lo = scale_pow2((float)l, e - 46 - lz);            // l 2^16 2^(e - 62 - lz)
    if (v < 0) {
        hi = -hi;
        lo = -lo;
    }
    const float s = hi + lo;
    return dfl(s, lo - (s - hi));
}

// Exponent e with 2^e above a nonnegative bound held as a float, read off its
// bits (FP32 and integer operations only: this part issues FP64 at 1/64 of the
// FP32 rate).  e is clamped to [-60, 100]: strengths are normalised (sum w^ =
// 1, y scaled to unit variance), so contributions below 2^(-60 - kBits) are
// negligible and bounds beyond 2^100 do not occur.
__device__ __forceinline__ signed char exponent_above(float bound)
{
    const int ex = (int)((__float_as_uint(bound) >> 23) & 0xFFu);   // 0 for zero (or subnormal)
    const int e = ex == 0 ? -60 : ex - 127 + 1;                     // bound < 2^(ex - 127 + 1)
    return (signed char)min(max(e, -60), 100);
}

// Grid exponent for a cell bound of maxbits (a float's bits) times count,
// the product rounded up.
__device__ __forceinline__ signed char row_exponent(unsigned maxbits, unsigned count)
{
    return exponent_above(__fmul_ru(__uint_as_float(maxbits), __uint2float_ru(count)));
}

// 2^(kBits - e), built from the exponent bits (the units are converted back by
// the FP32 path's first FFT stage and by fixed_to_dfl).
__device__ __forceinline__ float fixed_scale(float, int e)
{
    return __int_as_float((127 + Fixed<float>::kBits - e) << 23);
}
__device__ __forceinline__ double fixed_scale(double, int e)
{
    return __longlong_as_double((long long)(1023 + Fixed<double>::kBits - e) << 52);
}

// Exponent of the FP64 path's grid, one per block: every cell is a sum of at
// most `count` contributions each at most the series' largest strength
// component (smax bits); int64 leaves 62 bits below that bound, ample for it.
__device__ __forceinline__ signed char block_exponent(unsigned smax_bits, int count)
{
    return row_exponent(smax_bits, (unsigned)count);
}

// The FP32 path's per-row bound.  Each record adds q = ceil(|s| 2^16 / M) to
// its row (M: the series' largest strength component, so q <= 2^16; rounded
// up, so M q / 2^16 >= |s|), an integer sum whatever the order; a row's cells
// are then at most M qsum / 2^16, close to the sum of its records'
// magnitudes.  Rows of 65536 or more records (qsum could overflow) take
// M count instead.
__device__ __forceinline__ unsigned row_units(unsigned sbits, float inv_m)
{
    return __float2uint_ru(__fmul_ru(__uint_as_float(sbits), inv_m));
}
constexpr signed char kRowEmpty = kEmptyRow;   // row exponent of a row no record reaches
__device__ __forceinline__ signed char row_exponent_sum(unsigned m_bits, unsigned qsum,
                                                       unsigned count)
{
    if (count == 0) return kRowEmpty;
    const float m = __uint_as_float(m_bits);
    const float bound = count < 65536u ? __fmul_ru(m, __uint2float_ru(qsum)) * 0x1p-16f
                                       : __fmul_ru(m, __uint2float_ru(count));
    return exponent_above(bound);
}

// Footprint of a record (first covered cell a + N1 b) in the column block
// a0 .. a0 + BA - 1: the cells (cs + u, row), u < cnt, take kernel offsets
// i0 + u.  All of them lie in one row (b, or b + 1 where the footprint wraps
// past column N1 - 1): a block never holds both column N1 - 1 and column 0.
struct Foot {
    int i0, cs, cnt, row;
};
__device__ __forceinline__ Foot footprint(uint32_t ab, int a0, int BA, int N1, int N2, int w)
{
    const int aj = (int)(ab & 0xFFFFu);
    const int bj = (int)(ab >> 16);
    int o = aj - a0;
    if (o < 0) o += N1;
    Foot f;
    if (o < BA) { f.i0 = 0; f.cs = o; }
    else { f.i0 = N1 - o; f.cs = 0; }
    f.cnt = min(BA - f.cs, w - f.i0);
    f.row = bj + ((aj + f.i0 >= N1) ? 1 : 0);
    if (f.row >= N2) f.row -= N2;
    return f;
}

// ---------------------------------------------------------------------------
// Pass A: spread the block's points into BA columns of length N2 held in shared
// memory, FFT each column, multiply by exp(2 pi i a d / n) and store
// H[grid][d][a].  blockIdx.y selects the transform: 0 -> s1 (x), 1 -> s2 (x),
// 2 -> s3 (2x).
// ---------------------------------------------------------------------------
template <typename T>
struct PassAArgs {
    Geometry g;
    Batch bt;
    int shared;            // 1: the common s2 and s3 transforms of a shared-times batch
    int nofit;             // 1: the model has no offset; s2 is not needed
    PointSet<T> px, p2;
    const int *binstart;   // 2 * (nbins + 1)
    const Stats *st;       // per series: the strength maxima (FP64 grids)
    const Cplx<T> *twA;    // two-level root table, length N2
    const Cplx<T> *tw4;    // four-step table (lo 4096, hi)
    Cplx<T> *H;
    int cs;                // blocks per thread-block cluster along the columns (1: none)
    int ny;                // instances (transforms of series) along the grid's y
    int group;             // instances per block iteration of k_passA_group / k_passA_sh
    const T *cv;           // k_passA_sh: c_i of series s at cv[s * cstride + i] (sorted order)
    int64_t cstride;
};

template <typename T>
__device__ __forceinline__ T es_kernel(T z, T beta)
{
    const T s = sqrt(fmax(T(0), T(1) - z * z));
    return exp(beta * (s - T(1)));
}

// The ES kernel for the FP64 path in double-float arithmetic, on the FP32
// units (this part issues FP64 at 1/64 of the FP32 rate; the FP64 exp and
// sqrt were a fifth of the FP64 step).  s = sqrt(1 - z^2) from an FP32 root
// and one Newton correction; exp(x), x = beta (s - 1) in [-beta, 0], by the
// textbook reduction x = k ln 2 + r with |r| <= ln(2)/2 (ln 2 split into a
// 24-bit head and a tail, so k ln 2 is exact in double-float) and the Taylor
// series of exp(r) to degree 14 (remainder below 1e-18) by Horner's rule,
// then the exact scaling by 2^k.  Error up to about beta 2^-48 of the kernel's
// peak (1.3e-13 at beta = 30), checked on the device against the FP64
// evaluation (ls_selftest_kernel_eval); used for tolerances down to 1e-11.
__device__ __forceinline__ dfl dfl_fast_sum(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return dfl(s, b - (s - a));
}
__device__ double es_kernel_dfl(double z, dfl beta)
{
    const dfl zd(z);
    const dfl q = dfl(1.0f, 0.0f) - zd * zd;
    dfl s(0.0f, 0.0f);
    if (q.hi > 0.0f) {
        const float s0 = sqrtf(q.hi);
        const float p = s0 * s0;
        const float pe = fmaf(s0, s0, -p);                    // s0^2 = p + pe exactly
        const float rem = ((q.hi - p) - pe) + q.lo;           // q - s0^2
        s = dfl_fast_sum(s0, rem / (2.0f * s0));
    }
    const dfl x = beta * (s - dfl(1.0f, 0.0f));
    const float k = rintf(x.hi * 1.44269504088896341f);
    const float ln2_hi = 0.693145751953125f;                 // 24-bit head of ln 2 (exact k * ln2_hi)
    const float ln2_lo = 1.42860682030941723212e-6f;         // ln 2 - ln2_hi
    const dfl r = x - (dfl(k * ln2_hi, 0.0f) + dfl(k, 0.0f) * dfl(ln2_lo, 0.0f));
    // Taylor coefficients 1/n!, n = 14 .. 0
    const double c[15] = {1.0 / 87178291200.0, 1.0 / 6227020800.0, 1.0 / 479001600.0,
                          1.0 / 39916800.0, 1.0 / 3628800.0, 1.0 / 362880.0, 1.0 / 40320.0,
                          1.0 / 5040.0, 1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5,
                          1.0, 1.0};
    dfl e(c[0]);
#pragma unroll
    for (int i = 1; i < 15; ++i) e = e * r + dfl(c[i]);
    const int ki = (int)k;
    return (double)ldexpf(e.hi, ki) + (double)ldexpf(e.lo, ki);
}

// Self-test support: both evaluations of psi at n points of [-1, 1].
__global__ void k_kernel_eval_pair(int n, double beta, double *dfl_out, double *fp64_out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double z = -1.0 + 2.0 * (double)i / (double)(n - 1);
        dfl_out[i] = es_kernel_dfl(z, dfl(beta));
        fp64_out[i] = es_kernel(z, beta);
    }
}

// One instance (a transform of a series) of one column block; the tables are
// built when build_tables is set (the first instance a block takes).  kCluster:
// the launch pairs column blocks in clusters (A.cs > 1), the store path then.
template <typename T, bool kCluster, int kNC16 = 2>
__device__ __forceinline__ void passA_instance(const PassAArgs<T> &A, const int y,
                                               const bool build_tables)
{
    using V = Cplx<T>;               // storage: the spread's accumulators, H
    using F = typename FftOf<T>::type;   // the transform's type (double-float for FP64)
    static_assert(sizeof(F) == sizeof(V), "transform and storage types share the layout");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = A.g;
    const int N1 = g.N1, N2 = g.N2, BA = g.BA;
    const int Lp = padded_len(N2);
    const int nhi = (N2 + 63) >> 6;
    // The four-step twiddle tables cover the columns of the whole cluster
    // (tc = cs * BA from column a_base): the cluster store twiddles the
    // partner's columns as it writes them.
    const int rank = (int)(blockIdx.x % (unsigned)A.cs);
    const int tc = A.cs * BA;
    V *buf = reinterpret_cast<V *>(smem_raw);   // BA columns, padded layout
    F *bufF = reinterpret_cast<F *>(buf);       // the same columns once spread
    F *alo = bufF + (size_t)BA * Lp;            // W_n^{a dl}, dl < 64, per column
    const int nhiP = ahi_stride(nhi);
    F *ahi = alo + tc * kAloStride;             // W_n^{64 a dh}, per column
    F *roots = ahi + tc * nhiP;                 // two-level root table of length N2
    int *dtab = reinterpret_cast<int *>(roots + 64 + nhi);   // slot -> frequency table

    // Instance -> (series, transform 0: s1, 1: s2, 2: s3) and its slot of H.
    // Independent series: 3 per series.  Shared t and dy (the common transforms
    // of launch_shared_pipeline, instances 0 and 1): slots 0, 1 hold s2 and s3
    // of the common records.
    int ser, grid, slot;
    if (A.shared) {
        slot = y;
        ser = slot < 2 ? 0 : slot - 2;
        grid = slot < 2 ? slot + 1 : 0;
    } else {
        ser = y / 3;
        grid = y - 3 * ser;
        slot = y;
    }
    if (A.nofit && grid == 1) return;    // whole block: before any barrier (y is uniform)
    const int blk = blockIdx.x;
    const int a0 = blk * BA;
    const int a_base = (blk - rank) * BA;
    const int64_t pt_off = series_of(A.bt, ser).rec_off;

    // ---- spread set-up: the record ranges and each thread's first records are
    // requested before the prologue, so their latency overlaps it ----
    const PointSet<T> P = shifted((grid < 2) ? A.px : A.p2, pt_off);
    const V *str = (grid == 1) ? P.s[1] : P.s[0];
    const int *bs = A.binstart + (size_t)ser * 2 * (g.nbins + 1) + ((grid < 2) ? 0 : (g.nbins + 1));
    const int nbb = (g.w - 1 + BA - 1) >> g.logBA;   // bins before this one that reach it
    int r0s, r0e, r1s = 0, r1e = 0;
    if (nbb + 1 >= g.nbins) {
        r0s = bs[0];
        r0e = bs[g.nbins];
    } else if (blk - nbb >= 0) {
        r0s = bs[blk - nbb];
        r0e = bs[blk + 1];
    } else {
        r0s = bs[blk - nbb + g.nbins];
        r0e = bs[g.nbins];
        r1s = bs[0];
        r1e = bs[blk + 1];
    }
    const int cnt0 = r0e - r0s;
    const int total = cnt0 + (r1e - r1s);
    using I = typename Fixed<T>::I;
    // Per-row bounds of the fixed-point grids (FP32; pass 1 over the block's
    // records): count and strength units (row_units) of the records whose
    // footprint row is b, gathered with integer atomics (order-free) in the
    // column buffer before it is zeroed, then one exponent per row.  The FP64
    // grid takes one exponent for the block (block_exponent).
    uint32_t *rcnt = reinterpret_cast<uint32_t *>(smem_raw);    // N2 counts, N2 unit sums
    uint32_t *rmax = rcnt + N2;
    signed char *rexp = reinterpret_cast<signed char *>(dtab + (N2 >> g.fa.logRlast));
    for (int i = threadIdx.x; i < 2 * N2; i += blockDim.x) rcnt[i] = 0u;
    if (build_tables) {
        load_roots(roots, A.twA, N2);
        fill_slot_table(dtab, g.fa);
        for (int i = threadIdx.x; i < tc * 64; i += blockDim.x) {
            const int col = i >> 6;
            alo[col * kAloStride + (i & 63)] =
                to_fft(tw4_root(A.tw4, (int64_t)(a_base + col) * (i & 63)));
        }
        for (int i = threadIdx.x; i < tc * nhi; i += blockDim.x) {
            const int col = i / nhi;
            const int dh = i - col * nhi;
            ahi[col * nhiP + dh] =
                to_fft(tw4_root(A.tw4, mod_u32((int64_t)(a_base + col) * 64 * dh, g.n)));
        }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
        const unsigned mbits = A.st[ser].smax[grid];
        const float inv_m = __fdiv_ru(65536.0f, __uint_as_float(mbits));
        // kRow records per thread in flight at a time
        constexpr int kRow = 4;
        for (int e0 = threadIdx.x; e0 < total; e0 += kRow * blockDim.x) {
            uint32_t abq[kRow];
            V sq[kRow];
#pragma unroll
            for (int q = 0; q < kRow; ++q) {
                const int e = e0 + q * (int)blockDim.x;
                if (e < total) {
                    const int j = (e < cnt0) ? (r0s + e) : (r1s + e - cnt0);
                    abq[q] = __ldg(P.ab + j);
                    sq[q] = __ldg(str + j);
                }
            }
#pragma unroll
            for (int q = 0; q < kRow; ++q) {
                if (e0 + q * (int)blockDim.x >= total) break;
                const Foot f = footprint(abq[q], a0, BA, N1, N2, g.w);
                if (f.cnt <= 0) continue;
                atomicAdd(rcnt + f.row, 1u);
                atomicAdd(rmax + f.row, row_units(strength_bound_bits(sq[q]), inv_m));
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < N2; b += blockDim.x)
            rexp[b] = row_exponent_sum(mbits, rmax[b], rcnt[b]);
    } else {
        const signed char eb = block_exponent(A.st[ser].smax[grid], total);
        for (int b = threadIdx.x; b < N2; b += blockDim.x) rexp[b] = eb;
    }
    __syncthreads();
    I *ibuf = reinterpret_cast<I *>(buf);       // the columns as fixed-point pairs while spreading
    if constexpr (sizeof(T) == 4) {
        // only rows that records reach take additions; the conversion below
        // writes the others' zeros
        for (int b = threadIdx.x; b < N2; b += blockDim.x) {
            if (rexp[b] == kRowEmpty) continue;
            for (int col = 0; col < BA; ++col) {
                I *c = ibuf + 2 * ((size_t)col * Lp + pad16(b));
                c[0] = 0;
                c[1] = 0;
            }
        }
    } else {
        for (int i = threadIdx.x; i < 2 * BA * Lp; i += blockDim.x) ibuf[i] = 0;
    }
    // kPre records per thread are loaded before any is used, so their global
    // loads overlap instead of forming one dependent chain per record.
    constexpr int kPre = 4;
    uint32_t abv[kPre];
    T rv[kPre];
    V sv[kPre];
    auto load_chunk = [&](int e0) {
#pragma unroll
        for (int q = 0; q < kPre; ++q) {
            const int e = e0 + q * (int)blockDim.x;
            if (e < total) {
                const int j = (e < cnt0) ? (r0s + e) : (r1s + e - cnt0);
                abv[q] = __ldg(P.ab + j);
                rv[q] = __ldg(P.roff + j);
                sv[q] = __ldg(str + j);
            }
        }
    };
    load_chunk((int)threadIdx.x);
    __syncthreads();

    // ---- spread: each contribution rounded to its row's grid, added exactly ----
    const T halfw = T(0.5) * T(g.w);
    const T zscale = T(2) / T(g.w);
    const T beta = T(g.beta);
    const dfl beta_dfl(g.beta);
    // the double-float evaluation's error (measured up to 1.3e-13 of the peak
    // for beta <= 30: x = beta (s - 1) carries about beta 2^-48) stays about
    // a hundredth of the tolerances it serves; tighter ones evaluate in FP64
    const bool dfl_ok = g.eps >= 1e-11;
    for (int e0 = threadIdx.x; e0 < total; e0 += kPre * blockDim.x) {
        if (e0 != (int)threadIdx.x) load_chunk(e0);
#pragma unroll
        for (int q = 0; q < kPre; ++q) {
            if (e0 + q * (int)blockDim.x >= total) break;
            const Foot f = footprint(abv[q], a0, BA, N1, N2, g.w);
            if (f.cnt <= 0) continue;
            const T roff = rv[q];
            const T fs = fixed_scale(T(0), rexp[f.row]);
            const V s = mk2(sv[q].x * fs, sv[q].y * fs);     // exact: a power of two
            I *dst = ibuf + 2 * ((size_t)f.cs * Lp + pad16(f.row));
            for (int u = 0; u < f.cnt; ++u) {
                const T z = (roff - halfw + T(f.i0 + u)) * zscale;
                T v;
                if constexpr (sizeof(T) == 8) v = dfl_ok ? es_kernel_dfl(z, beta_dfl) : es_kernel(z, beta);
                else v = es_kernel(z, beta);
                Fixed<T>::add(dst, Fixed<T>::of(s.x * v));
                Fixed<T>::add(dst + 1, Fixed<T>::of(s.y * v));
                dst += 2 * (size_t)Lp;
            }
        }
    }
    __syncthreads();

    // ---- column FFTs over b.  FP32: the first stage reads the fixed-point
    // pairs, converts them with their rows' units and skips empty rows' loads.
    // FP64: convert in place first (same 16 bytes per cell) ----
    if constexpr (sizeof(T) == 4) {
        if ((BA & 1) == 0) fft_dif_fixed<2, kNC16>(bufF, BA, Lp, g.fa, roots, rexp, BA, 0);
        else fft_dif_fixed<1>(bufF, BA, Lp, g.fa, roots, rexp, BA, 0);
    } else {
        for (int col = 0; col < BA; ++col) {
            for (int b = threadIdx.x; b < N2; b += blockDim.x) {
                const size_t i = (size_t)col * Lp + pad16(b);
                bufF[i] = mk2(fixed_to_dfl(ibuf[2 * i], rexp[b]),
                              fixed_to_dfl(ibuf[2 * i + 1], rexp[b]));
            }
        }
        __syncthreads();
        fft_dif<1>(bufF, BA, Lp, g.fa, roots);
    }

    // ---- twiddle exp(2 pi i a d / n) and store H[grid][d][a], slot order ----
    if constexpr (kCluster) {
        // Cluster store.  A row of H receives only BA columns from one block,
        // so the cs blocks of a cluster (adjacent column blocks) write their
        // rows together: each block takes every cs-th row and writes the
        // cluster's cs * BA columns of it, twiddled, as 16-byte units, reading
        // the other blocks' columns from their shared memory, so each row
        // segment fills whole 32-byte sectors.
        namespace cg = cooperative_groups;
        cg::cluster_group cluster = cg::this_cluster();
        cluster.sync();
        const int cs = A.cs;
        const int cc = cs * BA;                                  // columns of the cluster
        constexpr int kPerUnit = 16 / (int)sizeof(V);            // columns per 16-byte unit
        const int ur = cc / kPerUnit;                            // units per row
        const int lr = ur < 32 ? ur : 32;                        // lanes per row
        const int rpw = 32 / lr;                                 // rows per warp step
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int sub_row = lane / lr, u0 = lane - sub_row * lr;
        F *Hc = reinterpret_cast<F *>(A.H + (size_t)slot * (size_t)g.n + (size_t)(blk - rank) * BA);
        // the block holding column c of the cluster: c / BA (its own columns are
        // read directly, the others through the cluster's shared-memory window)
        auto col_base = [&](int c) -> const F * {
            const int q = c / BA;
            return (q == rank ? bufF : cluster.map_shared_rank(bufF, q)) + (size_t)(c - q * BA) * Lp;
        };
        const int nwarps = (int)(blockDim.x >> 5);
        const int rows = (N2 - rank + cs - 1) / cs;               // rows this block writes
        const int step = nwarps * rpw;
        // kRows rows per lane at a time: their shared-memory reads across the
        // cluster are all in flight before the first store.
        constexpr int kRows = 4;
        for (int i0 = warp * rpw + sub_row; i0 < rows; i0 += kRows * step) {
            for (int u = u0; u < ur; u += lr) {
                F va[kRows], vb[kRows];
                int dd[kRows];
                const int c0 = sizeof(V) == 8 ? 2 * u : u, c1 = c0 + 1;
                const F *pa = col_base(c0);
                const F *pb = sizeof(V) == 8 ? col_base(c1) : pa;
#pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    const int i = i0 + r * step;
                    dd[r] = -1;
                    if (i < rows) {
                        const int pos = rank + cs * i;
                        dd[r] = slot_freq_tab(pos, dtab, g.fa);
                        const int sp = pad16(pos);
                        const int dl = dd[r] & 63, dh = dd[r] >> 6;
                        va[r] = cmul(pa[sp], cmul(alo[c0 * kAloStride + dl], ahi[c0 * nhiP + dh]));
                        if constexpr (sizeof(V) == 8)
                            vb[r] = cmul(pb[sp], cmul(alo[c1 * kAloStride + dl], ahi[c1 * nhiP + dh]));
                    }
                }
#pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    if (dd[r] < 0) continue;
                    F *dst = Hc + (size_t)dd[r] * N1;
                    if constexpr (sizeof(V) == 8)
                        reinterpret_cast<float4 *>(dst)[u] =
                            make_float4(va[r].x, va[r].y, vb[r].x, vb[r].y);
                    else
                        dst[u] = va[r];
                }
            }
        }
        cluster.sync();      // peers may still read this block's columns
        return;
    }
    F *H = reinterpret_cast<F *>(A.H + (size_t)slot * (size_t)g.n + a0);
    if constexpr (sizeof(T) == 4) {
        if ((BA & 1) == 0) {
            // Column pairs as one 16-byte store: a0, N1 and n are even, so every
            // pair starts on a 16-byte boundary.  A row of H receives only BA
            // columns from this block, so wider stores are not available here.
#pragma unroll 2
            for (int pos = threadIdx.x; pos < N2; pos += blockDim.x) {
                const int d = slot_freq_tab(pos, dtab, g.fa);
                const int sp = pad16(pos);
                float4 *dst = reinterpret_cast<float4 *>(H + (size_t)d * N1);
                for (int c0 = 0; c0 < BA; c0 += 2) {
                    const F t0 = cmul(alo[c0 * kAloStride + (d & 63)], ahi[c0 * nhiP + (d >> 6)]);
                    const F t1 = cmul(alo[(c0 + 1) * kAloStride + (d & 63)],
                                      ahi[(c0 + 1) * nhiP + (d >> 6)]);
                    const F v0 = cmul(bufF[(size_t)c0 * Lp + sp], t0);
                    const F v1 = cmul(bufF[(size_t)(c0 + 1) * Lp + sp], t1);
                    dst[c0 >> 1] = make_float4(v0.x, v0.y, v1.x, v1.y);
                }
            }
            return;
        }
    }
    for (int pos = threadIdx.x; pos < N2; pos += blockDim.x) {
        const int d = slot_freq_tab(pos, dtab, g.fa);
        const int sp = pad16(pos);
        F *dst = H + (size_t)d * N1;
        for (int col = 0; col < BA; ++col) {
            const F tw = cmul(alo[col * kAloStride + (d & 63)], ahi[col * nhiP + (d >> 6)]);
            dst[col] = cmul(bufF[(size_t)col * Lp + sp], tw);
        }
    }
}


// Pass A for many small grids of one batch launch of independent series: a
// block takes column block blk of `group` instances at a time (instances: the
// transforms of the series), their columns side by side in shared memory
// (member r owns columns r BA .. r BA + BA - 1), so the tables, the
// transforms' barriers and the stores are shared by the group.  No cluster
// pairs (small grids only).
constexpr int kMaxGroup = 8;   // instances per block iteration of the grouped kernels
// The grouped kernels run three blocks per SM (80 registers, at most
// kGroupSmemBudget bytes of grid rows per block): their per-barrier work is
// small, so more resident warps pay more than the registers the two-block
// form keeps (measured: uniform batch 139k -> 163k periodograms/s, ragged
// FP32 batch +8%, despite some register spills).
constexpr int kGroupBlocksPerSM = 3;
constexpr size_t kGroupSmemBudget = 66 * 1024;

template <typename T>
__global__ void __launch_bounds__(kThreadsA, kGroupBlocksPerSM) k_passA_group(PassAArgs<T> A)
{
    __shared__ int grp[4 * kMaxGroup + 1];
    __shared__ const uint32_t *g_ab[kMaxGroup];
    __shared__ const T *g_roff[kMaxGroup];
    __shared__ const Cplx<T> *g_str[kMaxGroup];
    __shared__ int g_slot[kMaxGroup];
    __shared__ signed char g_exp[kMaxGroup];   // FP64: one grid exponent per member
    __shared__ unsigned g_mbits[kMaxGroup];    // FP32: the member's strength maximum (bits)
    __shared__ float g_invm[kMaxGroup];        // and 2^16 over it, rounded up
    using V = Cplx<T>;
    using I = typename Fixed<T>::I;
    using F = typename FftOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = A.g;
    const int N1 = g.N1, N2 = g.N2, BA = g.BA;
    const int Lp = padded_len(N2);
    const int nhi = (N2 + 63) >> 6;
    const int G = A.group;
    V *buf = reinterpret_cast<V *>(smem_raw);
    F *bufF = reinterpret_cast<F *>(buf);
    F *alo = bufF + (size_t)G * BA * Lp;
    F *ahi = alo + BA * 64;
    F *roots = ahi + BA * nhi;
    int *dtab = reinterpret_cast<int *>(roots + 64 + nhi);
    const int blk = blockIdx.x;
    const int a0 = blk * BA;
    load_roots(roots, A.twA, N2);
    fill_slot_table(dtab, g.fa);
    for (int i = threadIdx.x; i < BA * 64; i += blockDim.x)
        alo[i] = to_fft(tw4_root(A.tw4, (int64_t)(a0 + (i >> 6)) * (i & 63)));
    for (int i = threadIdx.x; i < BA * nhi; i += blockDim.x) {
        const int col = i / nhi;
        ahi[i] = to_fft(tw4_root(A.tw4, mod_u32((int64_t)(a0 + col) * 64 * (i - col * nhi), g.n)));
    }
    const T halfw = T(0.5) * T(g.w);
    const T zscale = T(2) / T(g.w);
    const T beta = T(g.beta);
    const dfl beta_dfl(g.beta);
    const bool dfl_ok = g.eps >= 1e-11;
    const int nbb = (g.w - 1 + BA - 1) >> g.logBA;
    // instances taken here: every transform of every series, without the w^
    // grid when the model has no offset
    const int S = A.ny / 3;
    const int ni = A.nofit ? 2 * S : 3 * S;

    signed char *rexp = reinterpret_cast<signed char *>(dtab + (N2 >> g.fa.logRlast));   // G x N2

    for (int s0 = blockIdx.y * G; s0 < ni; s0 += gridDim.y * G) {
        const int gact = min(G, ni - s0);
        __syncthreads();                  // tables ready / the previous group is stored
        I *ibuf = reinterpret_cast<I *>(buf);   // fixed-point pairs while spreading
        // per-row bounds of member r: N2 counts and N2 max bits at the start of
        // its column region (before the region is zeroed for the spread)
        auto rows_of = [&](int r) {
            return reinterpret_cast<uint32_t *>(buf + (size_t)r * BA * Lp);
        };
        for (int r = 0; r < gact; ++r)
            for (int i = threadIdx.x; i < 2 * N2; i += blockDim.x) rows_of(r)[i] = 0u;
        // record ranges of the group's series (rows of grp: first range start,
        // its length, second range start, exclusive prefix of the totals)
        if ((int)threadIdx.x < gact) {
            const int r = threadIdx.x;
            const int idx = s0 + r;
            int ser, grid, slot;
            if (A.nofit) {
                ser = idx >> 1;
                grid = (idx & 1) ? 2 : 0;
                slot = 3 * ser + grid;
            } else {
                ser = idx / 3;
                grid = idx - 3 * ser;
                slot = idx;
            }
            const PointSet<T> P = shifted(grid < 2 ? A.px : A.p2, series_of(A.bt, ser).rec_off);
            g_ab[r] = P.ab;
            g_roff[r] = P.roff;
            g_str[r] = grid == 1 ? P.s[1] : P.s[0];
            g_slot[r] = slot;
            const int *bs = A.binstart + (size_t)ser * 2 * (g.nbins + 1) +
                            (grid < 2 ? 0 : (g.nbins + 1));
            int r0s, r0e, r1s = 0, r1e = 0;
            if (nbb + 1 >= g.nbins) {
                r0s = bs[0];
                r0e = bs[g.nbins];
            } else if (blk - nbb >= 0) {
                r0s = bs[blk - nbb];
                r0e = bs[blk + 1];
            } else {
                r0s = bs[blk - nbb + g.nbins];
                r0e = bs[g.nbins];
                r1s = bs[0];
                r1e = bs[blk + 1];
            }
            grp[4 * r] = r0s;
            grp[4 * r + 1] = r0e - r0s;
            grp[4 * r + 2] = r1s;
            grp[4 * r + 3] = (r0e - r0s) + (r1e - r1s);
            g_exp[r] = block_exponent(A.st[ser].smax[grid], grp[4 * r + 3]);
            g_mbits[r] = A.st[ser].smax[grid];
            g_invm[r] = __fdiv_ru(65536.0f, __uint_as_float(g_mbits[r]));
        }
        __syncthreads();
        if (threadIdx.x == 0) {           // prefix of the totals
            int acc = 0;
            for (int r = 0; r < gact; ++r) {
                const int tot = grp[4 * r + 3];
                grp[4 * r + 3] = acc;
                acc += tot;
            }
            grp[4 * kMaxGroup] = acc;
        }
        __syncthreads();
        const int all = grp[4 * kMaxGroup];
        // member and record index of the group's e-th record
        auto locate = [&](int e, int &r) {
            r = 0;
            while (r + 1 < gact && grp[4 * (r + 1) + 3] <= e) ++r;
            const int el = e - grp[4 * r + 3];
            return (el < grp[4 * r + 1]) ? grp[4 * r] + el : grp[4 * r + 2] + el - grp[4 * r + 1];
        };
        if constexpr (sizeof(T) == 4) {
            // pass 1: per-row counts and largest strength bounds (integer
            // atomics), kRow records per thread in flight
            constexpr int kRow = 4;
            for (int e0 = threadIdx.x; e0 < all; e0 += kRow * blockDim.x) {
                uint32_t abq[kRow];
                V sq[kRow];
                int rq[kRow];
#pragma unroll
                for (int q = 0; q < kRow; ++q) {
                    const int e = e0 + q * (int)blockDim.x;
                    rq[q] = -1;
                    if (e < all) {
                        int r;
                        const int j = locate(e, r);
                        abq[q] = __ldg(g_ab[r] + j);
                        sq[q] = __ldg(g_str[r] + j);
                        rq[q] = r;
                    }
                }
#pragma unroll
                for (int q = 0; q < kRow; ++q) {
                    if (rq[q] < 0) break;
                    const Foot f = footprint(abq[q], a0, BA, N1, N2, g.w);
                    if (f.cnt <= 0) continue;
                    uint32_t *rc = rows_of(rq[q]);
                    atomicAdd(rc + f.row, 1u);
                    atomicAdd(rc + N2 + f.row, row_units(strength_bound_bits(sq[q]), g_invm[rq[q]]));
                }
            }
            __syncthreads();
            for (int r = 0; r < gact; ++r) {
                const uint32_t *rc = rows_of(r);
                for (int b = threadIdx.x; b < N2; b += blockDim.x)
                    rexp[r * N2 + b] = row_exponent_sum(g_mbits[r], rc[N2 + b], rc[b]);
            }
        } else {
            for (int r = 0; r < gact; ++r)
                for (int b = threadIdx.x; b < N2; b += blockDim.x) rexp[r * N2 + b] = g_exp[r];
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            // only rows that records reach take additions (the conversion
            // writes the others' zeros)
            for (int r = 0; r < gact; ++r) {
                for (int b = threadIdx.x; b < N2; b += blockDim.x) {
                    if (rexp[r * N2 + b] == kRowEmpty) continue;
                    for (int col = 0; col < BA; ++col) {
                        I *c = ibuf + 2 * ((size_t)(r * BA + col) * Lp + pad16(b));
                        c[0] = 0;
                        c[1] = 0;
                    }
                }
            }
        } else {
            for (int i = threadIdx.x; i < 2 * gact * BA * Lp; i += blockDim.x) ibuf[i] = 0;
        }
        __syncthreads();
        // kPre records per thread in flight, over the group's records in turn
        constexpr int kPre = 4;
        for (int e0 = threadIdx.x; e0 < all; e0 += kPre * blockDim.x) {
            uint32_t abv[kPre];
            T rv[kPre];
            V sv[kPre];
            int rr[kPre];
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                const int e = e0 + q * (int)blockDim.x;
                rr[q] = -1;
                if (e < all) {
                    int r;
                    const int j = locate(e, r);
                    abv[q] = __ldg(g_ab[r] + j);
                    rv[q] = __ldg(g_roff[r] + j);
                    sv[q] = __ldg(g_str[r] + j);
                    rr[q] = r;
                }
            }
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                if (rr[q] < 0) break;
                const Foot f = footprint(abv[q], a0, BA, N1, N2, g.w);
                if (f.cnt <= 0) continue;
                const T fs = fixed_scale(T(0), rexp[rr[q] * N2 + f.row]);
                const V sq = mk2(sv[q].x * fs, sv[q].y * fs);     // exact: a power of two
                I *dst = ibuf + 2 * ((size_t)(rr[q] * BA + f.cs) * Lp + pad16(f.row));
                for (int u = 0; u < f.cnt; ++u) {
                    const T z = (rv[q] - halfw + T(f.i0 + u)) * zscale;
                    T v;
                    if constexpr (sizeof(T) == 8) v = dfl_ok ? es_kernel_dfl(z, beta_dfl) : es_kernel(z, beta);
                    else v = es_kernel(z, beta);
                    Fixed<T>::add(dst, Fixed<T>::of(sq.x * v));
                    Fixed<T>::add(dst + 1, Fixed<T>::of(sq.y * v));
                    dst += 2 * (size_t)Lp;
                }
            }
        }
        __syncthreads();
        // FP32: the first FFT stage converts the fixed-point pairs as it loads
        // (fft_dif_fixed); FP64: convert in place first
        if constexpr (sizeof(T) == 8) {
            for (int c = 0; c < gact * BA; ++c) {
                const signed char *re = rexp + (c / BA) * N2;
                for (int b = threadIdx.x; b < N2; b += blockDim.x) {
                    const size_t i = (size_t)c * Lp + pad16(b);
                    bufF[i] = mk2(fixed_to_dfl(ibuf[2 * i], re[b]),
                                  fixed_to_dfl(ibuf[2 * i + 1], re[b]));
                }
            }
            __syncthreads();
        }
        if constexpr (sizeof(T) == 4)
            fft_dif_fixed<2, 1>(bufF, gact * BA, Lp, g.fa, roots, rexp, BA, N2);
        else
            fft_dif<1>(bufF, gact * BA, Lp, g.fa, roots);
        // twiddle exp(2 pi i a d / n) and store H[2 + s][d][a], slot order; the
        // BA columns of a row go out as 16-byte units
        for (int pos = threadIdx.x; pos < N2; pos += blockDim.x) {
            const int d = slot_freq_tab(pos, dtab, g.fa);
            const int sp = pad16(pos);
            for (int r = 0; r < gact; ++r) {
                F *dst = reinterpret_cast<F *>(A.H + (size_t)g_slot[r] * (size_t)g.n +
                                               (size_t)d * N1 + a0);
                if constexpr (sizeof(F) == 8) {
                    for (int c0 = 0; c0 < BA; c0 += 2) {       // BA >= 2 (group launches)
                        const F v0 = cmul(bufF[(size_t)(r * BA + c0) * Lp + sp],
                                          cmul(alo[c0 * 64 + (d & 63)], ahi[c0 * nhi + (d >> 6)]));
                        const F v1 = cmul(bufF[(size_t)(r * BA + c0 + 1) * Lp + sp],
                                          cmul(alo[(c0 + 1) * 64 + (d & 63)],
                                               ahi[(c0 + 1) * nhi + (d >> 6)]));
                        reinterpret_cast<float4 *>(dst)[c0 >> 1] = make_float4(v0.x, v0.y, v1.x, v1.y);
                    }
                } else {
                    for (int col = 0; col < BA; ++col)
                        dst[col] = cmul(bufF[(size_t)(r * BA + col) * Lp + sp],
                                        cmul(alo[col * 64 + (d & 63)], ahi[col * nhi + (d >> 6)]));
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Shared-times batches (series with one time array and one dy: the batched
// mode of Sec. 2).  Positions, pre-phases and weights are the same for every
// series, so they are reduced, sorted and transformed once (the w^ transforms
// at f and 2f); a series contributes only its data: its weighted mean, its YY
// and one scalar per point, c_i = scale (y - ybar) at the i-th record of the
// common sorted order, from which pass A forms s1_i = c_i s2_i (s2 = w^ p, the
// common strength).  k_passA_sh then evaluates each record's kernel values
// once for a group of series.  Per-launch layout: Stats and tickets of series
// s at s (common: at S), partials reused kernel after kernel.
// ---------------------------------------------------------------------------

// Weights w_j = 1/dy_j^2 (FP64, kept for the series' sums), W = sum w_j into
// the common Stats entry, and the checks of t and dy.
__global__ void k_sh_weights(const double *__restrict__ t, const double *__restrict__ dy,
                             int64_t nd, double *wts, double *partials, unsigned int *counter,
                             Stats *stc, int *status)
{
    __shared__ double sh[32];
    const int64_t nch = (nd + kRedChunk - 1) / kRedChunk;
    bool ok = true;
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        double sw = 0.0;
        const int64_t j1 = min(nd, (c + 1) * kRedChunk);
        for (int64_t j = c * kRedChunk + threadIdx.x; j < j1; j += blockDim.x) {
            const double d = dy ? dy[j] : 1.0;
            ok &= finite_bits(d) && finite_bits(t[j]) && __double_as_longlong(d) > 0;
            const double w = rcp_fp64(d * d);
            wts[j] = w;
            sw += w;
        }
        const double a = block_sum(sw, sh);
        if (threadIdx.x == 0) partials[c] = a;
    }
    if (!ok) atomicOr(status, kStatBadInput);
    if (last_block(counter)) {
        double r[1];
        reduce_partials(partials, (int)nch, 1, r, sh);
        if (threadIdx.x == 0) {
            stc->W = r[0];
            stc->invW = 1.0 / r[0];
            stc->smax[0] = stc->smax[1] = stc->smax[2] = 0u;
            *counter = 0u;
        }
    }
}

// Common records: cells, kernel offsets and the strengths of the w^
// transforms (s2 = w^ p at x, s3 = w^ p^2 at 2x) from the exact phase
// reduction, formed as k_points forms them; the two grids' strength maxima.
template <typename T>
__global__ void k_sh_points(const double *__restrict__ t, int64_t nd, PhaseArgs ph, Geometry g,
                            const double *__restrict__ wts, PointSet<T> px, PointSet<T> p2,
                            Stats *stc)
{
    const double invW = stc->invW;
    unsigned m2 = 0u, m3 = 0u;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nd;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double tj = t[j];
        const double wh = wts[j] * invW;
        const u128 Fx = frac_fixed(ph.df_m, ph.df_e, 0, tj);
        const u128 Fc = frac_fixed(ph.f0_m, ph.f0_e, ph.f0_neg, tj) + (u128)(uint64_t)ph.K0 * Fx;
        uint32_t ab1, ab2;
        T r1, r2;
        split_fixed<T>(Fx, g, ab1, r1);
        split_fixed<T>(Fx << 1, g, ab2, r2);
        const Cplx<T> p = Cis<T>::of(Fc);
        const Cplx<T> q = Cis<T>::of(Fc << 1);
        const T wt = (T)wh;
        const Cplx<T> s2 = mk2(wt * p.x, wt * p.y), s3 = mk2(wt * q.x, wt * q.y);
        px.ab[j] = ab1;
        px.roff[j] = r1;
        px.s[1][j] = s2;
        p2.ab[j] = ab2;
        p2.roff[j] = r2;
        p2.s[0][j] = s3;
        m2 = max(m2, strength_bound_bits(s2));
        m3 = max(m3, strength_bound_bits(s3));
    }
    m2 = __reduce_max_sync(0xffffffffu, m2);
    m3 = __reduce_max_sync(0xffffffffu, m3);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stc->smax[1], m2);
        atomicMax(&stc->smax[2], m3);
    }
}

// Per series (blockIdx.y): WY = sum w_j y_j and WY2 = sum w_j y_j^2 with the
// common weights, then ybar and the strength scale as k_stats sets them.
__global__ void k_sh_stats(const double *__restrict__ y, Batch bt, const double *__restrict__ wts,
                           const Stats *stc, double *partials, unsigned int *counter, Stats *st,
                           int *status, int center)
{
    const int ser = blockIdx.y;
    const SeriesDesc sd = series_of(bt, ser);
    y += sd.y_off;
    const int64_t nd = sd.nd;
    const int64_t nch = (nd + kRedChunk - 1) / kRedChunk;
    partials += 3 * red_row0(sd.rec_off, ser);
    counter += 2 * ser;
    st += ser;
    __shared__ double sh[32];
    bool ok = true;
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        double swy = 0.0, swy2 = 0.0;
        const int64_t j1 = min(nd, (c + 1) * kRedChunk);
        for (int64_t j = c * kRedChunk + threadIdx.x; j < j1; j += blockDim.x) {
            const double yj = y[j];
            ok &= finite_bits(yj);
            const double wy = wts[j] * yj;
            swy += wy;
            swy2 = fma(wy, yj, swy2);
        }
        const double b = block_sum(swy, sh);
        const double q = block_sum(swy2, sh);
        if (threadIdx.x == 0) {
            partials[2 * c] = b;
            partials[2 * c + 1] = q;
        }
    }
    if (!ok) atomicOr(status, kStatBadInput);
    if (last_block(counter)) {
        double r[2];
        reduce_partials(partials, (int)nch, 2, r, sh);
        if (threadIdx.x == 0) {
            const double W = stc->W, WY = r[0], WY2 = r[1];
            st->W = W;
            st->WY = WY;
            st->WY2 = WY2;
            st->ybar = center ? WY / W : 0.0;
            st->invW = stc->invW;
            const double m2 = WY2 / W;
            const double var = fmax(m2 - st->ybar * st->ybar, 1e-20 * m2);
            st->scale = (var > 0.0 && isfinite(var)) ? 1.0 / sqrt(var) : 1.0;
            st->smax[0] = st->smax[1] = st->smax[2] = 0u;
            *counter = 0u;
        }
    }
}

// Per series (blockIdx.y): YY = sum w^_j (scale (y_j - ybar))^2 (FP64, the
// exact second pass, input order), and c_i = scale (y_perm(i) - ybar) in the
// common sorted order with the maximum of the s1 strength c_i s2_i as pass A
// forms it (the series' fixed-point grid bound).
template <typename T>
__global__ void k_sh_series(const double *__restrict__ y, Batch bt, const double *__restrict__ wts,
                            const int *__restrict__ perm, const Cplx<T> *__restrict__ s2sorted,
                            T *cvals, double *partials, unsigned int *counter, Stats *st,
                            int *status)
{
    const int ser = blockIdx.y;
    const SeriesDesc sd = series_of(bt, ser);
    y += sd.y_off;
    const int64_t nd = sd.nd;
    cvals += (size_t)ser * (size_t)nd;
    const int64_t nch = (nd + kRedChunk - 1) / kRedChunk;
    partials += 3 * red_row0(sd.rec_off, ser);
    counter += 2 * ser + 1;
    st += ser;
    __shared__ double sh[32];
    const double ybar = st->ybar, scale = st->scale;
    unsigned m1 = 0u;
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        double syy = 0.0;
        const int64_t j1 = min(nd, (c + 1) * kRedChunk);
        for (int64_t j = c * kRedChunk + threadIdx.x; j < j1; j += blockDim.x) {
            const double yc = y[j] - ybar;
            syy = fma(wts[j] * yc, yc, syy);
            const T cj = (T)(scale * (y[perm[j]] - ybar));   // j as a sorted index here
            cvals[j] = cj;
            const Cplx<T> s2 = s2sorted[j];
            m1 = max(m1, strength_bound_bits(mk2(cj * s2.x, cj * s2.y)));
        }
        const double a = block_sum(syy, sh);
        if (threadIdx.x == 0) partials[c] = a;
    }
    m1 = __reduce_max_sync(0xffffffffu, m1);
    if ((threadIdx.x & 31) == 0) atomicMax(&st->smax[0], m1);
    if (last_block(counter)) {
        double r[1];
        reduce_partials(partials, (int)nch, 1, r, sh);
        if (threadIdx.x == 0) {
            const double YY = r[0] * st->invW, Y2 = st->WY2 * st->invW;
            st->YY = YY * scale * scale;
            st->Y2 = Y2;
            finish_series_stats(st);
            // A constant series: variance zero up to the rounding of the mean.
            if (!(YY > 1e-24 * Y2)) atomicOr(status, kStatDegenerate);
            *counter = 0u;
        }
    }
}

// Pass A for the series grids of a shared-times batch: a block takes column
// block blk of `group` series at a time (member r owns columns r BA .. r BA +
// BA - 1, its s1 grid in H slot 2 + r of the chunk).  The series share the
// records, so each record's footprint and kernel values are computed once and
// applied to every member's strength c_i s2_i; the row counts are common and
// the strength units per member (FP32 fixed-point grids).  No cluster pairs.
// kKv: bound of min(BA, w), the cells of a record in the block's columns
// (8 for tiles of up to 8 columns, else 16), the kernel values kept in registers.
template <typename T, int kKv>
__global__ void __launch_bounds__(kThreadsA, kGroupBlocksPerSM) k_passA_sh(PassAArgs<T> A)
{
    using V = Cplx<T>;
    using F = typename FftOf<T>::type;
    using I = typename Fixed<T>::I;
    __shared__ unsigned g_mbits[kMaxGroup];    // members' strength maxima (bits)
    __shared__ float g_invm[kMaxGroup];        // and 2^16 over them, rounded up
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = A.g;
    const int N1 = g.N1, N2 = g.N2, BA = g.BA;
    const int Lp = padded_len(N2);
    const int nhi = (N2 + 63) >> 6;
    const int G = A.group;
    V *buf = reinterpret_cast<V *>(smem_raw);
    F *bufF = reinterpret_cast<F *>(buf);
    F *alo = bufF + (size_t)G * BA * Lp;
    F *ahi = alo + BA * 64;
    F *roots = ahi + BA * nhi;
    int *dtab = reinterpret_cast<int *>(roots + 64 + nhi);
    signed char *rexp = reinterpret_cast<signed char *>(dtab + (N2 >> g.fa.logRlast));   // G x N2
    const int blk = blockIdx.x;
    const int a0 = blk * BA;
    load_roots(roots, A.twA, N2);
    fill_slot_table(dtab, g.fa);
    for (int i = threadIdx.x; i < BA * 64; i += blockDim.x)
        alo[i] = to_fft(tw4_root(A.tw4, (int64_t)(a0 + (i >> 6)) * (i & 63)));
    for (int i = threadIdx.x; i < BA * nhi; i += blockDim.x) {
        const int col = i / nhi;
        ahi[i] = to_fft(tw4_root(A.tw4, mod_u32((int64_t)(a0 + col) * 64 * (i - col * nhi), g.n)));
    }
    const T halfw = T(0.5) * T(g.w);
    const T zscale = T(2) / T(g.w);
    const T beta = T(g.beta);
    const dfl beta_dfl(g.beta);
    const bool dfl_ok = g.eps >= 1e-11;
    // the block's records (common to all series): bins blk - nbb .. blk of geometry x
    const PointSet<T> P = A.px;
    const int *bs = A.binstart;
    const int nbb = (g.w - 1 + BA - 1) >> g.logBA;
    int r0s, r0e, r1s = 0, r1e = 0;
    if (nbb + 1 >= g.nbins) {
        r0s = bs[0];
        r0e = bs[g.nbins];
    } else if (blk - nbb >= 0) {
        r0s = bs[blk - nbb];
        r0e = bs[blk + 1];
    } else {
        r0s = bs[blk - nbb + g.nbins];
        r0e = bs[g.nbins];
        r1s = bs[0];
        r1e = bs[blk + 1];
    }
    const int cnt0 = r0e - r0s;
    const int total = cnt0 + (r1e - r1s);
    const V *s2r = P.s[1];
    const int S = A.ny;
    // member r's grid region holds, before it is zeroed for the spread, the
    // common row counts (member 0) and the member's row strength units
    auto rows_of = [&](int r) { return reinterpret_cast<uint32_t *>(buf + (size_t)r * BA * Lp); };

    for (int s0 = blockIdx.y * G; s0 < S; s0 += gridDim.y * G) {
        const int gact = min(G, S - s0);
        const T *cv = A.cv + (size_t)s0 * A.cstride;     // member r: cv + r * cstride
        __syncthreads();                  // tables ready / the previous group is stored
        for (int i = threadIdx.x; i < N2; i += blockDim.x) rows_of(0)[i] = 0u;
        for (int r = 0; r < gact; ++r)
            for (int i = threadIdx.x; i < N2; i += blockDim.x) rows_of(r)[N2 + i] = 0u;
        if ((int)threadIdx.x < gact) {
            const int r = threadIdx.x;
            g_mbits[r] = A.st[s0 + r].smax[0];
            g_invm[r] = __fdiv_ru(65536.0f, __uint_as_float(g_mbits[r]));
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            // pass 1: common row counts, per-member strength units
            constexpr int kRow = 4;
            for (int e0 = threadIdx.x; e0 < total; e0 += kRow * blockDim.x) {
                uint32_t abq[kRow];
                V sq[kRow];
                int jq[kRow];
#pragma unroll
                for (int q = 0; q < kRow; ++q) {
                    const int e = e0 + q * (int)blockDim.x;
                    jq[q] = -1;
                    if (e < total) {
                        const int j = (e < cnt0) ? (r0s + e) : (r1s + e - cnt0);
                        abq[q] = __ldg(P.ab + j);
                        sq[q] = __ldg(s2r + j);
                        jq[q] = j;
                    }
                }
#pragma unroll
                for (int q = 0; q < kRow; ++q) {
                    if (jq[q] < 0) break;
                    const Foot f = footprint(abq[q], a0, BA, N1, N2, g.w);
                    if (f.cnt <= 0) continue;
                    atomicAdd(rows_of(0) + f.row, 1u);
                    for (int r = 0; r < gact; ++r) {
                        const T c = __ldg(cv + (size_t)r * A.cstride + jq[q]);
                        atomicAdd(rows_of(r) + N2 + f.row,
                                  row_units(strength_bound_bits(mk2(c * sq[q].x, c * sq[q].y)),
                                            g_invm[r]));
                    }
                }
            }
            __syncthreads();
            for (int r = 0; r < gact; ++r)
                for (int b = threadIdx.x; b < N2; b += blockDim.x)
                    rexp[r * N2 + b] = row_exponent_sum(g_mbits[r], rows_of(r)[N2 + b], rows_of(0)[b]);
        } else {
            for (int r = 0; r < gact; ++r) {
                const signed char eb = block_exponent(g_mbits[r], total);
                for (int b = threadIdx.x; b < N2; b += blockDim.x) rexp[r * N2 + b] = eb;
            }
        }
        __syncthreads();
        I *ibuf = reinterpret_cast<I *>(buf);
        if constexpr (sizeof(T) == 4) {
            for (int r = 0; r < gact; ++r) {
                for (int b = threadIdx.x; b < N2; b += blockDim.x) {
                    if (rexp[r * N2 + b] == kRowEmpty) continue;
                    for (int col = 0; col < BA; ++col) {
                        I *c = ibuf + 2 * ((size_t)(r * BA + col) * Lp + pad16(b));
                        c[0] = 0;
                        c[1] = 0;
                    }
                }
            }
        } else {
            for (int i = threadIdx.x; i < 2 * gact * BA * Lp; i += blockDim.x) ibuf[i] = 0;
        }
        __syncthreads();
        // spread: a record's kernel values once, then every member's strength
        constexpr int kPre = 2;
        for (int e0 = threadIdx.x; e0 < total; e0 += kPre * blockDim.x) {
            uint32_t abv[kPre];
            T rv[kPre];
            V sv[kPre];
            int jv[kPre];
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                const int e = e0 + q * (int)blockDim.x;
                jv[q] = -1;
                if (e < total) {
                    const int j = (e < cnt0) ? (r0s + e) : (r1s + e - cnt0);
                    abv[q] = __ldg(P.ab + j);
                    rv[q] = __ldg(P.roff + j);
                    sv[q] = __ldg(s2r + j);
                    jv[q] = j;
                }
            }
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                if (jv[q] < 0) break;
                const Foot f = footprint(abv[q], a0, BA, N1, N2, g.w);
                if (f.cnt <= 0) continue;
                T kv[kKv];
#pragma unroll
                for (int u = 0; u < kKv; ++u) {
                    if (u < f.cnt) {
                        const T z = (rv[q] - halfw + T(f.i0 + u)) * zscale;
                        if constexpr (sizeof(T) == 8) kv[u] = dfl_ok ? es_kernel_dfl(z, beta_dfl) : es_kernel(z, beta);
                        else kv[u] = es_kernel(z, beta);
                    }
                }
                for (int r = 0; r < gact; ++r) {
                    const T c = __ldg(cv + (size_t)r * A.cstride + jv[q]);
                    const V s1 = mk2(c * sv[q].x, c * sv[q].y);
                    const T fs = fixed_scale(T(0), rexp[r * N2 + f.row]);
                    const V sq = mk2(s1.x * fs, s1.y * fs);     // exact: a power of two
                    I *dst = ibuf + 2 * ((size_t)(r * BA + f.cs) * Lp + pad16(f.row));
#pragma unroll
                    for (int u = 0; u < kKv; ++u) {
                        if (u < f.cnt) {
                            Fixed<T>::add(dst, Fixed<T>::of(sq.x * kv[u]));
                            Fixed<T>::add(dst + 1, Fixed<T>::of(sq.y * kv[u]));
                            dst += 2 * (size_t)Lp;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if constexpr (sizeof(T) == 8) {
            for (int c = 0; c < gact * BA; ++c) {
                const signed char *re = rexp + (c / BA) * N2;
                for (int b = threadIdx.x; b < N2; b += blockDim.x) {
                    const size_t i = (size_t)c * Lp + pad16(b);
                    bufF[i] = mk2(fixed_to_dfl(ibuf[2 * i], re[b]),
                                  fixed_to_dfl(ibuf[2 * i + 1], re[b]));
                }
            }
            __syncthreads();
        }
        if constexpr (sizeof(T) == 4)
            fft_dif_fixed<2, 1>(bufF, gact * BA, Lp, g.fa, roots, rexp, BA, N2);
        else
            fft_dif<1>(bufF, gact * BA, Lp, g.fa, roots);
        // twiddle exp(2 pi i a d / n) and store H[2 + s][d][a], slot order
        for (int pos = threadIdx.x; pos < N2; pos += blockDim.x) {
            const int d = slot_freq_tab(pos, dtab, g.fa);
            const int sp = pad16(pos);
            for (int r = 0; r < gact; ++r) {
                F *dst = reinterpret_cast<F *>(A.H + (size_t)(2 + s0 + r) * (size_t)g.n +
                                               (size_t)d * N1 + a0);
                if constexpr (sizeof(F) == 8) {
                    if ((BA & 1) == 0) {
                        for (int c0 = 0; c0 < BA; c0 += 2) {
                            const F v0 = cmul(bufF[(size_t)(r * BA + c0) * Lp + sp],
                                              cmul(alo[c0 * 64 + (d & 63)], ahi[c0 * nhi + (d >> 6)]));
                            const F v1 = cmul(bufF[(size_t)(r * BA + c0 + 1) * Lp + sp],
                                              cmul(alo[(c0 + 1) * 64 + (d & 63)],
                                                   ahi[(c0 + 1) * nhi + (d >> 6)]));
                            reinterpret_cast<float4 *>(dst)[c0 >> 1] =
                                make_float4(v0.x, v0.y, v1.x, v1.y);
                        }
                        continue;
                    }
                }
                for (int col = 0; col < BA; ++col)
                    dst[col] = cmul(bufF[(size_t)(r * BA + col) * Lp + sp],
                                    cmul(alo[col * 64 + (d & 63)], ahi[col * nhi + (d >> 6)]));
            }
        }
    }
}

// One instance per block (blockIdx.y), the usual launch (two blocks per SM:
// with three, 80 registers, small grids ran 4-12% slower).  kThr threads per
// block: the FP32 path takes kThreadsAWide.
template <typename T, bool kCluster, int kThr = kThreadsA, int kMinB = 2>
__global__ void __launch_bounds__(kThr, kMinB) k_passA(PassAArgs<T> A)
{
    // blocks compiled for 80 registers take the radix-16 stages one column at
    // a time (fewer live values; on the 1.9e7-cell grid 0.647 -> 0.637 ms)
    constexpr int kNC16 = (kThr > kThreadsA && sizeof(T) == 4) ? 1 : 2;
    passA_instance<T, kCluster, kNC16>(A, (int)blockIdx.y, true);
}

// Many instances per block: y = blockIdx.y, + gridDim.y, ... of the block's
// column block (a persistent loop when a batch has more instances than the
// launch has rows of blocks); the tables depend only on the columns and are
// built once.  An instance skipped without a fitted mean is skipped by the
// whole block (and cluster), so the barriers stay uniform.
// kMinB: blocks per SM the registers are sized for (2: 128 registers; 3: 80,
// launched only where the shared memory lets three blocks share an SM, see
// blocks_per_sm).
template <typename T, bool kCluster, int kMinB>
__global__ void __launch_bounds__(kThreadsA, kMinB) k_passA_loop(PassAArgs<T> A)
{
    bool first = true;
    for (int y = blockIdx.y; y < A.ny; y += gridDim.y) {
        if (A.nofit) {
            const int grid = y % 3;
            if (grid == 1) continue;
        }
        if (!first) __syncthreads();      // the previous instance is done with the buffer
        passA_instance<T, kCluster, (kMinB >= 3 && sizeof(T) == 4) ? 1 : 2>(A, y, first);
        first = false;
    }
}

// ---------------------------------------------------------------------------
// Power.  Generalised (floating-mean) periodogram, standard normalisation,
// from the six sums and YY.  With CC = sum w^ cos^2 - C^2 = (1 + C2)/2 - C^2,
// SS = (1 - C2)/2 - S^2, CS = S2/2 - C S, the rotation through w tau
// (tan 2 w tau = (S2 - 2CS)/(C2 - (C^2 - S^2))) diagonalises M = [[CC, CS],
// [CS, SS]], so YC_tau^2/CC_tau + YS_tau^2/SS_tau = v^T M^-1 v with v = (Ch, Sh):
// P = (Ch^2 SS - 2 Ch Sh CS + Sh^2 CC) / ((CC SS - CS^2) YY).
// ---------------------------------------------------------------------------

// Explicit tau rotation (FP64), used for a nearly singular M (all phases equal
// mod pi): a vanishing CC_tau or SS_tau term is dropped.
__device__ __noinline__ double ls_power_tau(double Ch, double Sh, double C, double S, double C2, double S2,
                               double YY, double lam_tol)
{
    const double num = S2 - 2.0 * C * S;
    const double den = C2 - (C * C - S * S);
    const double r = hypot(num, den);
    double c2 = 1.0, s2 = 0.0;
    if (r > 0.0) {
        c2 = den / r;
        s2 = num / r;
    }
    double c, s;
    if (c2 >= 0.0) {
        c = sqrt(0.5 * (1.0 + c2));
        s = s2 / (2.0 * c);
    } else {
        s = sqrt(0.5 * (1.0 - c2));
        if (s2 < 0.0) s = -s;
        c = s2 / (2.0 * s);
    }
    const double YC = Ch * c + Sh * s;
    const double YS = Sh * c - Ch * s;
    const double Ct = C * c + S * s;
    const double St = S * c - C * s;
    const double CCt = 0.5 * (1.0 + C2 * c2 + S2 * s2) - Ct * Ct;
    const double SSt = 0.5 * (1.0 - C2 * c2 - S2 * s2) - St * St;
    double p = 0.0;
    if (CCt > lam_tol) p += YC * YC / CCt;
    if (SSt > lam_tol) p += YS * YS / SSt;
    return p / YY;
}

__device__ __forceinline__ double ls_power_fp64(double Ch, double Sh, double C, double S,
                                                double C2, double S2, double YY, double lam_tol)
{
    const double CC = 0.5 * (1.0 + C2) - C * C;
    const double SS = 0.5 * (1.0 - C2) - S * S;
    const double CS = 0.5 * S2 - C * S;
    const double D = CC * SS - CS * CS;
    // D = lam_min lam_max and CC + SS = lam_min + lam_max: the closed form needs
    // lam_min clearly above the sums' accuracy.
    if (D > lam_tol * (CC + SS) && CC > 0.0 && SS > 0.0) {
        const double N = Ch * Ch * SS - 2.0 * Ch * Sh * CS + Sh * Sh * CC;
        return N / (D * YY);
    }
    return ls_power_tau(Ch, Sh, C, S, C2, S2, YY, lam_tol);
}

// Double-float ("float-float") arithmetic: a value is hi + lo with |lo| <=
// ulp(hi)/2, about 48 significant bits.  Error-free transforms: Knuth's
// two-sum, the fast two-sum for |a| >= |b|, and the fma two-product.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
// Sum with Dekker's add (no second renormalisation): error below about
// 2^-47 (|x| + |y|), the error model of an FP64 add of the same operands (2^-53
// (|x| + |y|)) at 48 bits.  The ratio's inputs are FP32 sums whose own errors
// scale with the same magnitudes, so a bound relative to |x + y| (the longer
// two-sum-of-low-parts form) buys nothing here.
__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const ff p = two_prod(x.hi, y.hi);
    return fast_two_sum(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}
// x / y: the float quotient q1 = x.hi / y.hi, corrected by the remainder
// x - q1 y formed exactly up to the low parts (q1 y.hi = p exactly by the fma
// two-product, and x.hi - p.hi is exact since p.hi is within a few ulp of
// x.hi): relative error about 2^-45.
__device__ __forceinline__ ff ff_div(ff x, ff y)
{
    const float ry = __frcp_rn(y.hi);
    const float q1 = x.hi * ry;
    const ff p = two_prod(q1, y.hi);
    const float r = fmaf(-q1, y.lo, ((x.hi - p.hi) - p.lo) + x.lo);
    return fast_two_sum(q1, r * ry);
}

// hi + lo rounded to the nearest double, on the integer pipe (hl_to_double).
__device__ __forceinline__ double ff_to_double(ff p) { return hl_to_double(p.hi, p.lo); }

// FP32 path: the sums arrive as FP32 values (exact inputs here); the ratio is
// evaluated in double-float, whose rounding (~1e-13 of the terms' magnitudes)
// is far below the FP32 sums' own error, and falls back to FP64 for a nearly
// singular M.  The terms of M (from C, S, C2, S2) are formed apart from those
// of the data (Ch, Sh), so series that share their times share them.
struct PowerM {
    ff CC, SS, CS, D;
    float C, S, C2, S2;
    bool regular;          // the closed form applies (M clearly nonsingular)
};
__device__ __forceinline__ PowerM power_m_ff(float C, float S, float C2, float S2, float lam_tol)
{
    PowerM m;
    m.C = C;
    m.S = S;
    m.C2 = C2;
    m.S2 = S2;
    m.CC = ff_add(two_sum(0.5f, 0.5f * C2), ff_neg(two_prod(C, C)));
    m.SS = ff_add(two_sum(0.5f, -0.5f * C2), ff_neg(two_prod(S, S)));
    m.CS = ff_add(ff{0.5f * S2, 0.f}, ff_neg(two_prod(C, S)));
    m.D = ff_add(ff_mul(m.CC, m.SS), ff_neg(ff_mul(m.CS, m.CS)));
    m.regular = m.D.hi > lam_tol * (m.CC.hi + m.SS.hi) && m.CC.hi > 0.f && m.SS.hi > 0.f;
    return m;
}
__device__ __forceinline__ double power_data_ff(const PowerM &m, float Ch, float Sh, ff YY,
                                                double YYd, float lam_tol)
{
    if (!m.regular) return ls_power_tau(Ch, Sh, m.C, m.S, m.C2, m.S2, YYd, (double)lam_tol);
    const ff ChSh = two_prod(Ch, Sh);
    const ff N = ff_add(ff_add(ff_mul(two_prod(Ch, Ch), m.SS), ff_mul(two_prod(Sh, Sh), m.CC)),
                        ff_neg(ff_mul(ff{2.f * ChSh.hi, 2.f * ChSh.lo}, m.CS)));
    return ff_to_double(ff_div(N, ff_mul(m.D, YY)));
}
__device__ __forceinline__ double ls_power_ff(float Ch, float Sh, float C, float S, float C2,
                                              float S2, ff YY, double YYd, float lam_tol)
{
    return power_data_ff(power_m_ff(C, S, C2, S2, lam_tol), Ch, Sh, YY, YYd, lam_tol);
}

// FP64 path at tolerances of 1e-11 and above: the transforms deliver
// double-float values, and the deconvolution and the ratio stay in double-float
// on the FP32 units (rounding about 2^-46 of the terms' magnitudes, far below
// the sums' own error of eps); the same ratio in FP64 took 40% of pass B on a
// part whose FP64 rate is 1/64 of its FP32 rate (1.9e7-cell grid: 1.04 of
// 2.65 ms).  A nearly singular M takes the FP64 rotation form.
__device__ __noinline__ ff double_to_ff_fp64(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}
// A double as a double-float on the integer pipe: hi takes the top 24 bits of
// the significand, lo the remaining 29 bits rounded to 24 (relative error
// below 2^-48), then renormalised.  Exponents within 2^+-70 of 1 (the
// deconvolution factors); others take the FP64 conversions out of line.
__device__ __forceinline__ ff double_to_ff(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 1023 - 70 || e > 1023 + 70) return double_to_ff_fp64(x);
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const float hi = __uint_as_float(sgn | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
    float lo = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull)) *
               __uint_as_float((unsigned)(e - 1023 - 52 + 127) << 23);
    if (sgn) lo = -lo;
    return fast_two_sum(hi, lo);
}
__device__ __noinline__ double power_dfl_singular(ff Ch, ff Sh, ff C, ff S, ff C2, ff S2, double YY,
                                                  double lam_tol)
{
    return ls_power_fp64(ff_to_double(Ch), ff_to_double(Sh), ff_to_double(C), ff_to_double(S),
                         ff_to_double(C2), ff_to_double(S2), YY, lam_tol);
}
__device__ __forceinline__ ff ff_half(ff x) { return {0.5f * x.hi, 0.5f * x.lo}; }   // exact
__device__ __forceinline__ double ls_power_dfl(dfl2 a1, dfl2 a2, dfl2 a3, double dc, ff YY,
                                               double YYd, float lam_tol, double lam_told)
{
    const ff d = double_to_ff(dc);
    const ff Ch = ff_mul(ff{a1.x.hi, a1.x.lo}, d), Sh = ff_mul(ff{a1.y.hi, a1.y.lo}, d);
    const ff C = ff_mul(ff{a2.x.hi, a2.x.lo}, d), S = ff_mul(ff{a2.y.hi, a2.y.lo}, d);
    const ff C2 = ff_mul(ff{a3.x.hi, a3.x.lo}, d), S2 = ff_mul(ff{a3.y.hi, a3.y.lo}, d);
    const ff hc2 = ff_half(C2);
    const ff CC = ff_add(ff_add(ff{0.5f, 0.f}, hc2), ff_neg(ff_mul(C, C)));
    const ff SS = ff_add(ff_add(ff{0.5f, 0.f}, ff_neg(hc2)), ff_neg(ff_mul(S, S)));
    const ff CS = ff_add(ff_half(S2), ff_neg(ff_mul(C, S)));
    const ff D = ff_add(ff_mul(CC, SS), ff_neg(ff_mul(CS, CS)));
    if (!(D.hi > lam_tol * (CC.hi + SS.hi) && CC.hi > 0.f && SS.hi > 0.f))
        return power_dfl_singular(Ch, Sh, C, S, C2, S2, YYd, lam_told);
    const ff ChSh = ff_mul(Ch, Sh);
    const ff N = ff_add(ff_add(ff_mul(ff_mul(Ch, Ch), SS), ff_mul(ff_mul(Sh, Sh), CC)),
                        ff_neg(ff_mul(ff{2.f * ChSh.hi, 2.f * ChSh.lo}, CS)));
    return ff_to_double(ff_div(N, ff_mul(D, YY)));
}

// ---------------------------------------------------------------------------
// Pass B: for row d, FFT the three grids over a (length N1), deconvolve the
// needed modes and evaluate the power.
// ---------------------------------------------------------------------------
template <typename T>
struct PassBArgs {
    Geometry g;
    Batch bt;
    int shared;            // see PassAArgs
    // 0: the three rows of each series.  Shared times: 1 transforms the two
    // common rows (w^ at f and 2f, H slots 0 and 1) once and writes them back
    // deconvolved, in slot order; 2 (k_passB_series) then transforms the
    // series' own rows and reads the common values from there.
    int stage;
    const Cplx<T> *twB;    // two-level root table, length N1
    Cplx<T> *H;
    const T *deconv;       // 1/phi_hat(|k'|) in pass-B order, [d * N1 + slot]
    const Stats *st;
    double *power;
    double *sums;
    double lam_tol;        // eigenvalues of M at or below this count as zero
    int nofit;             // 1: no offset in the model: C = S = 0, grid s2 absent
    int norm;              // 0 standard, 1 model, 2 log, 3 psd
    int nser;              // series of the launch (stages 0 and 2)
    int group;             // series per block of k_passB_series / k_passB_group
};

// Normalisation of the standard power P = p / YY (p the explained weighted
// sum of squares with w^): model p / (YY - p) = P / (1 - P); log -ln(1 - P);
// psd p W / 2 = P YY W / 2 with the unscaled YY and W = sum w.
// The FP32 path's log keeps FP32 relative accuracy over the whole range
// without an FP64 logarithm: log1p(-P) for P < 1/2 (no cancellation in 1 - P
// for small P), and the log of 1 - P, formed exactly in FP64, above.
// The model, log and psd forms out of line (with them inline, the standard
// form's hot loop issued their FP64 work predicated: pass B of the 1.9e7-cell
// grid 0.449 against 0.422 ms).
template <typename T>
__device__ __noinline__ double ls_normalise_other(double P, int norm, double psd_factor)
{
    switch (norm) {
    case 1: return P * rcp_fp64(1.0 - P);
    case 2:
        if (sizeof(T) == 4)
            return P < 0.5 ? -(double)log1pf(-(float)P) : -(double)logf((float)(1.0 - P));
        return -log1p(-P);
    case 3: return P * psd_factor;
    default: return P;
    }
}
template <typename T>
__device__ __forceinline__ double ls_normalise(double P, int norm, double psd_factor)
{
    return norm == 0 ? P : ls_normalise_other<T>(P, norm, psd_factor);
}

// Asynchronous global -> shared copies of one complex element (sm_80+):
// 8 bytes (FP32 complex) through L1, 16 bytes (FP64 complex) bypassing it.
__device__ __forceinline__ void cp_async_elem(float2 *dst, const float2 *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s),
                 "l"((unsigned long long)__cvta_generic_to_global(src)) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2 *dst, const double2 *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s),
                 "l"((unsigned long long)__cvta_generic_to_global(src)) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// Wait until every committed copy of this thread has landed (a hardware wait on
// the thread's own copies; the block barrier that follows publishes them).
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T> struct PowerOut;

template <> struct PowerOut<double> {
    __device__ __forceinline__ static double eval(double2 g1, double2 g2, double2 g3, double dc,
                                                  double YY, ff, double lam_tol) {
        return ls_power_fp64(g1.x * dc, g1.y * dc, g2.x * dc, g2.y * dc, g3.x * dc, g3.y * dc,
                             YY, lam_tol);
    }
};
template <> struct PowerOut<float> {
    __device__ __forceinline__ static double eval(float2 g1, float2 g2, float2 g3, float dc,
                                                  double YY, ff YYf, float lam_tol) {
        return ls_power_ff(g1.x * dc, g1.y * dc, g2.x * dc, g2.y * dc, g3.x * dc, g3.y * dc,
                           YYf, YY, lam_tol);
    }
};

// The eigenvalue tolerance of M in the types the power evaluations take,
// converted once per block (an FP64 conversion per mode would run on the slow
// FP64 pipe).
template <typename T>
struct LamTol {
    double d;
    T t;
    float f;
    __device__ __forceinline__ explicit LamTol(double x) : d(x), t((T)x), f((float)x) {}
};

// The power of one mode from its transform values a1, a2, a3 (a2 null without
// a fitted mean: C = S = 0) and its deconvolution factor: FP32 grids through
// PowerOut; FP64 grids in double-float where the tolerance allows (dfl_power)
// and through PowerOut in FP64 below it.  Every pass-B kernel of independent
// series evaluates a mode through this, so a series has the same bits alone
// and in a batch.
template <typename T>
__device__ __forceinline__ double mode_power(const typename FftOf<T>::type &a1,
                                             const typename FftOf<T>::type *a2,
                                             const typename FftOf<T>::type &a3, T dc, double YY,
                                             ff YYf, const LamTol<T> &lt, bool dfl_power)
{
    using V = Cplx<T>;
    if constexpr (sizeof(T) == 8) {
        if (dfl_power) {
            const dfl2 z = {dfl(0.f, 0.f), dfl(0.f, 0.f)};
            return ls_power_dfl(a1, a2 ? *a2 : z, a3, dc, YYf, YY, lt.f, lt.d);
        }
    }
    const V g1 = from_fft(a1), g3 = from_fft(a3);
    const V g2 = a2 ? from_fft(*a2) : mk2(T(0), T(0));
    return PowerOut<T>::eval(g1, g2, g3, dc, YY, YYf, lt.t);
}

// kStage is PassBArgs::stage as a template parameter: each launch carries only
// its own code (fewer instruction-fetch stalls than one kernel for all stages).
// kThr: threads per block; above kThreadsB the row transforms deal their
// (row, butterfly) pairs to all threads (more warps per SM where shared memory
// allows only two blocks).
template <typename T, int kStage, int kMinB, int kThr = kThreadsB>
__global__ void __launch_bounds__(kThr, kMinB) k_passB(PassBArgs<T> B)
{
    using V = Cplx<T>;
    using F = typename FftOf<T>::type;   // the transform's type (double-float for FP64)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = B.g;
    const int N1 = g.N1, N2 = g.N2;
    const int Lp = padded_len(N1);
    F *buf = reinterpret_cast<F *>(smem_raw);   // 3 rows, padded layout
    F *roots = buf + 3 * (size_t)Lp;            // two-level root table of length N1
    int *dtab = reinterpret_cast<int *>(roots + 64 + ((N1 + 63) >> 6));
    const int d = blockIdx.x;
    constexpr int stage = kStage;
    // radix-16 stages one transform at a time in the 80-register (three blocks
    // per SM) form: two at a time held 64 values and spilled
    constexpr int kNC16B = kMinB >= 3 ? 1 : 2;
    load_roots(roots, B.twB, N1);
    fill_slot_table(dtab, g.fb);
    static_assert(stage == 0 || stage == 1, "stage 2 runs in k_passB_series");
    const int nser = stage == 1 ? 1 : B.nser;

    // The block takes the series s = blockIdx.y, + gridDim.y, ... of its row d
    // (a persistent loop when the batch has more series than the launch has
    // rows of blocks): the tables are built once.
    for (int ser = blockIdx.y; ser < nser; ser += gridDim.y) {
    const SeriesDesc sd = series_of(B.bt, ser);
    const int64_t nf = sd.nf, K0 = sd.ph.K0;
    const Stats *stat = B.st + ser;
    double *power = B.power ? B.power + sd.out_off : nullptr;
    double *sums = B.sums ? B.sums + 6 * sd.out_off : nullptr;
    __syncthreads();                      // the previous series is done with buf
    // rows of H straight into shared memory with asynchronous copies: every
    // element of the three rows is in flight at once, without registers.
    for (int gi = 0; gi < 3; ++gi) {
        if (B.nofit && gi == 1) continue;
        if (stage == 1 && gi == 0) continue;
        const size_t slot = B.shared ? (gi == 0 ? 2 + ser : gi - 1) : 3 * ser + gi;
        const V *src = B.H + slot * (size_t)g.n + (size_t)d * N1;
        V *dst = reinterpret_cast<V *>(buf + (size_t)gi * Lp);   // H holds F bits (pass A)
        for (int i = threadIdx.x; i < N1; i += blockDim.x) cp_async_elem(dst + pad16(i), src + i);
    }
    cp_async_commit();
    // per-series scalars, loaded while the copies run
    const double YY = stat->YY;
    const double psd_factor = stat->psd;
    const double unscale = stat->unscale;
    cp_async_wait_all();
    __syncthreads();

    if constexpr (stage == 1) {             // rows 1 and 2 (row 2 alone without a fitted mean)
        if (B.nofit) fft_dif<1>(buf + 2 * (size_t)Lp, 1, Lp, g.fb, roots);
        else if (sizeof(T) == 4) fft_dif<2, kNC16B>(buf + Lp, 2, Lp, g.fb, roots);
        else fft_dif<1>(buf + Lp, 2, Lp, g.fb, roots);
        // write both rows back deconvolved, in slot order, over the same row d of
        // H slots 0 and 1 (this block read that row; no other block touches it)
        V *o2 = B.H + (size_t)d * N1;
        V *o3 = B.H + (size_t)g.n + (size_t)d * N1;
        const T *dcr = B.deconv + (size_t)d * N1;
        for (int pos = threadIdx.x; pos < N1; pos += blockDim.x) {
            const T dc = __ldg(dcr + pos);
            const int sp = pad16(pos);
            o2[pos] = B.nofit ? mk2(T(0), T(0)) : cscale(from_fft(buf[Lp + sp]), dc);
            o3[pos] = cscale(from_fft(buf[2 * Lp + sp]), dc);
        }
        continue;
    }
    if constexpr (kThr > kThreadsB) {
        if (B.nofit) fft_dif_dealt(buf, 2, 2 * Lp, g.fb, roots);   // rows 0 and 2
        else fft_dif_dealt(buf, 3, Lp, g.fb, roots);
    } else if (B.nofit) {                   // rows 0 and 2
        if (sizeof(T) == 4) fft_dif<2, kNC16B>(buf, 2, 2 * Lp, g.fb, roots);
        else fft_dif<1>(buf, 2, 2 * Lp, g.fb, roots);
    } else {
        if (sizeof(T) == 4) fft_dif<3, kNC16B>(buf, 3, Lp, g.fb, roots);
        else fft_dif<1>(buf, 3, Lp, g.fb, roots);
    }

    const bool dfl_power = g.eps >= 1e-11;   // FP64 path: the ratio in double-float
    const LamTol<T> lt(B.lam_tol);
    ff YYf;
    YYf.hi = stat->yy_hi;
    YYf.lo = stat->yy_lo;
    const int64_t n = g.n;
    const int64_t hi_start = n - K0;       // k >= hi_start -> k' = k - n < 0
    const int64_t lo_end = nf - K0;        // k <  lo_end   -> k' = k >= 0
    const int c1 = (lo_end > d) ? div_u32(lo_end - d + N2 - 1, N2) : 0;
    const int c2 = div_u32(hi_start - d + N2 - 1, N2);
    // kDc deconvolution factors per thread are loaded (coalesced, pass-B order)
    // before any is used, so their latency is paid once per group.
    constexpr int kDc = 4;
    const T *dcrow = B.deconv + (size_t)d * N1;
    for (int p0 = threadIdx.x; p0 < N1; p0 += kDc * blockDim.x) {
        T dcv[kDc];
#pragma unroll
        for (int r = 0; r < kDc; ++r) {
            const int pos = p0 + r * (int)blockDim.x;
            dcv[r] = pos < N1 ? __ldg(dcrow + pos) : T(0);
        }
#pragma unroll
        for (int r = 0; r < kDc; ++r) {
            const int pos = p0 + r * (int)blockDim.x;
            if (pos >= N1) break;
            const int c = slot_freq_tab(pos, dtab, g.fb);
            if (c >= c1 && c < c2) continue;            // mode not requested
            const int64_t k = d + (int64_t)N2 * c;
            const int64_t kp = (c < c1) ? k : k - n;
            const int sp = pad16(pos);
            const T dc = dcv[r];
            const int64_t out = kp + K0;
            if (power) {
                const double P = mode_power<T>(buf[sp], B.nofit ? nullptr : &buf[Lp + sp],
                                               buf[2 * Lp + sp], dc, YY, YYf, lt, dfl_power);
                power[out] = ls_normalise<T>(P, B.norm, psd_factor);
            }
            if (sums) {
                const V g1 = from_fft(buf[sp]), g3 = from_fft(buf[2 * Lp + sp]);
                const V g2 = B.nofit ? mk2(T(0), T(0)) : from_fft(buf[Lp + sp]);
                // Ch, Sh were formed from scale * (y - ybar): report them unscaled.
                double *o = sums + 6 * out;
                o[0] = (double)(g1.x * dc) * unscale; o[1] = (double)(g1.y * dc) * unscale;
                o[2] = (double)(g2.x * dc); o[3] = (double)(g2.y * dc);
                o[4] = (double)(g3.x * dc); o[5] = (double)(g3.y * dc);
            }
        }
    }
    }   // series
}

// ---------------------------------------------------------------------------
// Pass B for the series of a shared-times batch (after stage 1 wrote the common
// rows back deconvolved): a block takes row d of `group` series at a time, their
// rows side by side in shared memory next to the two common rows, so the row
// copies, the transforms' barriers, the common values and the deconvolution
// factor of each mode are shared by the group.  All series have the same grid.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreadsB, kGroupBlocksPerSM) k_passB_series(PassBArgs<T> B)
{
    using V = Cplx<T>;
    using F = typename FftOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = B.g;
    const int N1 = g.N1, N2 = g.N2;
    const int Lp = padded_len(N1);
    const int G = B.group;
    F *buf = reinterpret_cast<F *>(smem_raw);   // rows 0, 1: common values; 2 .. 1+G: series
    V *bufV = reinterpret_cast<V *>(buf);
    F *roots = buf + (size_t)(2 + G) * Lp;
    double *sc = reinterpret_cast<double *>(roots + 64 + ((N1 + 63) >> 6));   // 4 per series
    int64_t *soff = reinterpret_cast<int64_t *>(sc + 4 * G);                   // output offsets
    int *dtab = reinterpret_cast<int *>(soff + G);
    const int d = blockIdx.x;
    load_roots(roots, B.twB, N1);
    fill_slot_table(dtab, g.fb);
    for (int pos = threadIdx.x; pos < N1; pos += blockDim.x) {
        const int sp = pad16(pos);
        bufV[sp] = B.H[(size_t)d * N1 + pos];
        bufV[Lp + sp] = B.H[(size_t)g.n + (size_t)d * N1 + pos];
    }
    const SeriesDesc sd0 = series_of(B.bt, 0);
    const int64_t nf = sd0.nf, K0 = sd0.ph.K0;
    const int64_t n = g.n;
    const int c1 = (nf - K0 > d) ? div_u32(nf - K0 - d + N2 - 1, N2) : 0;
    const int c2 = div_u32(n - K0 - d + N2 - 1, N2);
    const T lam_tol_t = (T)B.lam_tol;
    const T *dcrow = B.deconv + (size_t)d * N1;

    for (int s0 = blockIdx.y * G; s0 < B.nser; s0 += gridDim.y * G) {
        const int gact = min(G, B.nser - s0);
        __syncthreads();                  // the previous group is done with its rows
        for (int r = 0; r < gact; ++r) {
            const V *src = B.H + (size_t)(2 + s0 + r) * (size_t)n + (size_t)d * N1;
            V *dst = bufV + (size_t)(2 + r) * Lp;
            for (int i = threadIdx.x; i < N1; i += blockDim.x) cp_async_elem(dst + pad16(i), src + i);
        }
        cp_async_commit();
        if ((int)threadIdx.x < gact) {
            const int r = threadIdx.x;
            const Stats *stat = B.st + s0 + r;
            const double YY = stat->YY;
            sc[4 * r] = YY;
            sc[4 * r + 1] = stat->psd;
            // the YY pair's float bits (read per mode without FP64 conversions)
            float *yyp = reinterpret_cast<float *>(sc + 4 * r + 2);
            yyp[0] = stat->yy_hi;
            yyp[1] = stat->yy_lo;
            soff[r] = series_of(B.bt, s0 + r).out_off;
        }
        cp_async_wait_all();
        __syncthreads();
        if (sizeof(T) == 4) fft_dif<2, 1>(buf + 2 * (size_t)Lp, gact, Lp, g.fb, roots);
        else fft_dif<1>(buf + 2 * (size_t)Lp, gact, Lp, g.fb, roots);

        for (int pos = threadIdx.x; pos < N1; pos += blockDim.x) {
            const int c = slot_freq_tab(pos, dtab, g.fb);
            if (c >= c1 && c < c2) continue;            // mode not requested
            const int64_t k = d + (int64_t)N2 * c;
            const int64_t out = ((c < c1) ? k : k - n) + K0;
            const int sp = pad16(pos);
            const T dc = __ldg(dcrow + pos);
            const V g2 = bufV[sp], g3 = bufV[Lp + sp];
            if constexpr (sizeof(T) == 4) {
                // the terms of M are the same for every series of the group
                const PowerM m = power_m_ff(g2.x, g2.y, g3.x, g3.y, lam_tol_t);
                for (int r = 0; r < gact; ++r) {
                    const V g1 = cscale(from_fft(buf[(size_t)(2 + r) * Lp + sp]), dc);
                    const float2 yyp = *reinterpret_cast<const float2 *>(sc + 4 * r + 2);
                    const ff YYf = {yyp.x, yyp.y};
                    const double P = power_data_ff(m, g1.x, g1.y, YYf, sc[4 * r], lam_tol_t);
                    B.power[soff[r] + out] = ls_normalise<T>(P, B.norm, sc[4 * r + 1]);
                }
            } else {
                for (int r = 0; r < gact; ++r) {
                    const V g1 = cscale(from_fft(buf[(size_t)(2 + r) * Lp + sp]), dc);
                    const float2 yyp = *reinterpret_cast<const float2 *>(sc + 4 * r + 2);
                    const ff YYf = {yyp.x, yyp.y};
                    const double P = PowerOut<T>::eval(g1, g2, g3, T(1), sc[4 * r], YYf, lam_tol_t);
                    B.power[soff[r] + out] = ls_normalise<T>(P, B.norm, sc[4 * r + 1]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Pass B for many small grids of independent series (stage 0 of a batch whose
// series all have this grid): a block takes row d of `group` series at a time,
// their rows (s1, s2, s3 each; s1, s3 without a fitted mean) side by side in
// shared memory, so the tables, the copies' wait, the transforms' barriers and
// the deconvolution factors are shared by the group.  The series share the
// grid but not N_f or the first mode K0.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreadsB, kGroupBlocksPerSM) k_passB_group(PassBArgs<T> B)
{
    using V = Cplx<T>;
    using F = typename FftOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = B.g;
    const int N1 = g.N1, N2 = g.N2;
    const int logN1 = 31 - __clz(N1);
    const int Lp = padded_len(N1);
    const int G = B.group;
    const int nr = B.nofit ? 2 : 3;              // rows per series; s3 is the last
    F *buf = reinterpret_cast<F *>(smem_raw);    // series r: rows nr r .. nr r + nr - 1
    V *bufV = reinterpret_cast<V *>(buf);
    F *roots = buf + (size_t)nr * G * Lp;
    double *sc = reinterpret_cast<double *>(roots + 64 + ((N1 + 63) >> 6));   // 4 per series
    int64_t *obase = reinterpret_cast<int64_t *>(sc + 4 * G);   // out_off + K0 per series
    int *cr = reinterpret_cast<int *>(obase + G);               // c1, c2 per series
    int *dtab = cr + 2 * G;
    const int d = blockIdx.x;
    const int64_t n = g.n;
    load_roots(roots, B.twB, N1);
    fill_slot_table(dtab, g.fb);
    const bool dfl_power = g.eps >= 1e-11;   // FP64 path: the ratio in double-float
    const LamTol<T> lt(B.lam_tol);
    const T *dcrow = B.deconv + (size_t)d * N1;

    for (int s0 = blockIdx.y * G; s0 < B.nser; s0 += gridDim.y * G) {
        const int gact = min(G, B.nser - s0);
        __syncthreads();                  // tables ready / the previous group is done
        // row d of every grid of the group, flattened over (row, element)
        for (int e = threadIdx.x; e < gact * nr * N1; e += blockDim.x) {
            const int row = e >> logN1, i = e & (N1 - 1);
            const int r = row / nr, j = row - nr * r;
            const int gi = (B.nofit && j == 1) ? 2 : j;
            const V *src = B.H + (size_t)(3 * (s0 + r) + gi) * (size_t)n + (size_t)d * N1;
            cp_async_elem(bufV + (size_t)row * Lp + pad16(i), src + i);
        }
        cp_async_commit();
        if ((int)threadIdx.x < gact) {
            const int r = threadIdx.x;
            const SeriesDesc sd = series_of(B.bt, s0 + r);
            const Stats *stat = B.st + s0 + r;
            const double YY = stat->YY;
            sc[4 * r] = YY;
            sc[4 * r + 1] = stat->psd;
            // the YY pair's float bits (read per mode without FP64 conversions)
            float *yyp = reinterpret_cast<float *>(sc + 4 * r + 2);
            yyp[0] = stat->yy_hi;
            yyp[1] = stat->yy_lo;
            const int64_t nf = sd.nf, K0 = sd.ph.K0;
            cr[2 * r] = (nf - K0 > d) ? (int)((nf - K0 - d + N2 - 1) / N2) : 0;
            cr[2 * r + 1] = (int)((n - K0 - d + N2 - 1) / N2);
            obase[r] = sd.out_off + K0;
        }
        cp_async_wait_all();
        __syncthreads();
        if (sizeof(T) == 4) fft_dif<2, 1>(buf, gact * nr, Lp, g.fb, roots);
        else fft_dif<1>(buf, gact * nr, Lp, g.fb, roots);

        for (int e = threadIdx.x; e < gact * N1; e += blockDim.x) {
            const int r = e >> logN1, pos = e & (N1 - 1);
            const int c = slot_freq_tab(pos, dtab, g.fb);
            const int c1 = cr[2 * r], c2 = cr[2 * r + 1];
            if (c >= c1 && c < c2) continue;            // mode not requested
            const int64_t k = d + (int64_t)N2 * c;
            const int64_t kp = (c < c1) ? k : k - n;
            const int sp = pad16(pos);
            const T dc = __ldg(dcrow + pos);
            const size_t base = (size_t)nr * r * Lp + sp;
            const float2 yyp = *reinterpret_cast<const float2 *>(sc + 4 * r + 2);
            const ff YYf = {yyp.x, yyp.y};
            const double P = mode_power<T>(buf[base], B.nofit ? nullptr : &buf[base + Lp],
                                           buf[base + (size_t)(nr - 1) * Lp], dc, sc[4 * r], YYf,
                                           lt, dfl_power);
            B.power[obase[r] + kp] = ls_normalise<T>(P, B.norm, sc[4 * r + 1]);
        }
    }
}

// ---------------------------------------------------------------------------
// Deconvolution table: 1/phi_hat(k), phi_hat(k) = w int_0^1 psi(z) cos(pi k w z / n) dz
// by the plan's quadrature rule (nodes z, weights already times psi(z)).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_deconv(T *out, int64_t count, double w_over_n, double w, const double *z,
                         const double *wpsi, int q)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        const double kk = (double)k * w_over_n;
        for (int i = 0; i < q; ++i) s += wpsi[i] * cospi(kk * z[i]);
        out[k] = (T)(1.0 / (w * s));
    }
}

template <typename T>
__global__ void k_deconv_slot(T *out, const T *__restrict__ compact, int64_t count, Geometry g)
{
    const int logN1 = 31 - __clz(g.N1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = i >> logN1;
        const int pos = (int)(i & (g.N1 - 1));
        const int64_t k = d + (int64_t)g.N2 * slot_to_freq(pos, g.fb);
        const int64_t m = k < g.n - k ? k : g.n - k;
        out[i] = m < count ? compact[m] : T(0);
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers
// ---------------------------------------------------------------------------
template <typename T>
size_t point_record_bytes()
{
    return 2 * sizeof(uint32_t) + sizeof(T) + 2 * sizeof(Cplx<T>);
}

// Blocks of a pass kernel whose dynamic shared memory is smem that fit one
// SM's shared memory (228 KB, 1 KB reserved per block).  Where three fit, the
// loop form of pass A and pass B are launched compiled for three blocks per SM
// (80 registers): on GB300 that ran ragged batches 4-7% and pass B of 3.7e5-
// and 4.7e6-cell grids 8-14% faster; where only two fit, the 128-register form
// keeps its registers (pass B of a 1.9e7-cell grid ran 6% slower with 80).
static int blocks_per_sm(size_t smem)
{
    return (int)((size_t)228 * 1024 / (smem + 1024));
}

// Columns, per-column and root tables, slot table, and one exponent byte per
// row (the spread's per-row fixed-point grids).
size_t passA_smem_bytes(const Geometry &g, size_t cx, int cs)
{
    const size_t nhi = (size_t)(g.N2 + 63) / 64;
    return cx * ((size_t)g.BA * padded_len(g.N2) +
                 (size_t)cs * g.BA * (kAloStride + ahi_stride((int)nhi)) + 64 + nhi) +
           sizeof(int) * (size_t)(g.N2 / g.fa.Rlast) + (size_t)g.N2;
}

size_t passB_smem_bytes(const Geometry &g, size_t cx)
{
    return cx * (3 * (size_t)padded_len(g.N1) + 64 + (size_t)(g.N1 + 63) / 64) +
           sizeof(int) * (size_t)(g.N1 / g.fb.Rlast);
}

// Series rows per block of k_passB_series: as many as fit (with the two common
// rows) in the grouped kernels' shared-memory budget, at most 8.
static int passB_group(const Geometry &g, size_t cx)
{
    const size_t row = cx * (size_t)padded_len(g.N1);
    const size_t budget = kGroupSmemBudget;
    int G = (int)(budget / row) - 2;
    return G < 1 ? 1 : (G > 8 ? 8 : G);
}

// Series per block of k_passB_group: as many as fit (nr rows each) in the
// grouped kernels' shared-memory budget, at most 8.
static int passB_group_indep(const Geometry &g, size_t cx, int nr)
{
    const size_t row = cx * (size_t)padded_len(g.N1);
    const int G = (int)(kGroupSmemBudget / (row * nr));
    return G > 8 ? 8 : G;
}

static size_t passB_group_smem_bytes(const Geometry &g, size_t cx, int G, int nr)
{
    return cx * ((size_t)nr * G * padded_len(g.N1) + 64 + (size_t)(g.N1 + 63) / 64) +
           (4 * sizeof(double) + sizeof(int64_t) + 2 * sizeof(int)) * (size_t)G +
           sizeof(int) * (size_t)(g.N1 / g.fb.Rlast);
}

static size_t passB_series_smem_bytes(const Geometry &g, size_t cx, int G)
{
    return cx * ((size_t)(2 + G) * padded_len(g.N1) + 64 + (size_t)(g.N1 + 63) / 64) +
           (4 * sizeof(double) + sizeof(int64_t)) * (size_t)G +
           sizeof(int) * (size_t)(g.N1 / g.fb.Rlast);
}

template <typename T>
static PointSet<T> carve(void *base, int64_t max_nd)
{
    PointSet<T> p;
    char *b = static_cast<char *>(base);
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    p.s[0] = reinterpret_cast<Cplx<T> *>(b + off);
    off = align(off + sizeof(Cplx<T>) * (size_t)max_nd);
    p.s[1] = reinterpret_cast<Cplx<T> *>(b + off);
    off = align(off + sizeof(Cplx<T>) * (size_t)max_nd);
    p.roff = reinterpret_cast<T *>(b + off);
    off = align(off + sizeof(T) * (size_t)max_nd);
    p.ab = reinterpret_cast<uint32_t *>(b + off);
    off = align(off + sizeof(uint32_t) * (size_t)max_nd);
    p.rank = reinterpret_cast<uint32_t *>(b + off);
    return p;
}

void decompose_double(double x, uint64_t &m, int &e, int &neg)
{
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    neg = (int)(b >> 63);
    const int ex = (int)((b >> 52) & 0x7ff);
    m = (b & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull);
    e = (ex ? ex : 1) - 1075;
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per (kernel, device) for the whole process.  The limit only permits:
// occupancy follows the size each launch asks for, so one setting serves every
// plan, and no thread can lower it under another's launch.
static cudaError_t allow_max_dynamic_smem(const void *fn)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &d : done)
        if (d.first == fn && d.second == dev) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    done.emplace_back(fn, dev);
    return cudaSuccess;
}

// Launch k_passA (one instance per block) with cfg's grid, shared memory and
// cluster attribute: FP32 blocks of kThreadsAWide threads, FP64 blocks of
// kThreadsAF64 (compiled for one block per SM when wider than kThreadsA: the
// FP64 columns leave room for one).
template <typename T>
static cudaError_t launch_passA_single(cudaLaunchConfig_t cfg, int cs, const PassAArgs<T> &A)
{
    constexpr int kThr = sizeof(T) == 4 ? kThreadsAWide : kThreadsAF64;
    constexpr int kMinB = (sizeof(T) == 8 && kThr > kThreadsA) ? 1 : 2;
    cudaError_t err;
    if ((err = allow_max_dynamic_smem((const void *)k_passA<T, false, kThr, kMinB>)) !=
            cudaSuccess ||
        (err = allow_max_dynamic_smem((const void *)k_passA<T, true, kThr, kMinB>)) != cudaSuccess)
        return err;
    cfg.blockDim = dim3(kThr);
    return cs > 1 ? cudaLaunchKernelEx(&cfg, k_passA<T, true, kThr, kMinB>, A)
                  : cudaLaunchKernelEx(&cfg, k_passA<T, false, kThr, kMinB>, A);
}

// Kernels launch_pipeline has enqueued (or recorded into graphs) in this process.
static std::atomic<long long> g_pipeline_kernels{0};

long long pipeline_kernel_count() { return g_pipeline_kernels.load(std::memory_order_relaxed); }

template <typename T>
cudaError_t launch_pipeline(const Geometry &g, const Workspace &ws, int64_t capacity,
                            const Batch &bt, int64_t max_nd, const double *t, const double *y,
                            const double *dy, double *power, double *sums, int nred,
                            cudaStream_t st, cudaEvent_t *ev, int mode)
{
    int nk = 6;    // kernels enqueued: stats, points, rank, chunk scan, scan, scatter, then the passes
    const int nofit = (mode & kModeNoFit) ? 1 : 0;
    const int center = (!nofit || !(mode & kModeNoCenter)) ? 1 : 0;
    cudaError_t err;
    const int S = bt.S;
    PointSet<T> rx = carve<T>(ws.pts_raw[0], capacity), r2 = carve<T>(ws.pts_raw[1], capacity);
    PointSet<T> sx = carve<T>(ws.pts_sorted[0], capacity), s2 = carve<T>(ws.pts_sorted[1], capacity);

    int nsm = 0, dev_id = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_id);
    if (nsm <= 0) nsm = 152;
    if (ev) cudaEventRecord(ev[0], st);
    k_stats<<<dim3(nred, S), 256, 0, st>>>(t, y, dy, bt, ws.partials, ws.counter, ws.stats,
                                           ws.status, center, ws.wts);
    k_points<T><<<dim3(nred, S), 256, 0, st>>>(t, y, ws.wts, bt, g, rx, r2, ws.partials, ws.counter,
                                               ws.stats, ws.status);
    if (ev) cudaEventRecord(ev[1], st);
    // stable ranks and chunk histograms: at most one block per chunk of the
    // largest series, at most about eight blocks per SM over the launch
    {
        const size_t smR = sizeof(unsigned short) * 2 * (kThreadsPts / 32) * (size_t)g.nbins;
        if ((err = allow_max_dynamic_smem((const void *)k_rank)) != cudaSuccess) return err;
        int64_t nrk = (max_nd + kChunk - 1) / kChunk;
        const int64_t cap = (8 * (int64_t)nsm + S - 1) / S;
        if (nrk > cap) nrk = cap;
        k_rank<<<dim3((unsigned)nrk, S), kThreadsPts, smR, st>>>(bt, g, rx.ab, r2.ab, rx.rank,
                                                               ws.chist);
    }
    k_chunk_scan<<<dim3((2 * g.nbins + 31) / 32, S), 256, 0, st>>>(bt, g.nbins, ws.chist, ws.hist);
    k_scan<<<S, 1024, 0, st>>>(ws.hist, g.nbins, ws.binstart);
    int nsc = (int)((max_nd + 255) / 256);
    if (nsc > 4096) nsc = 4096;
    k_scatter<T><<<dim3(nsc, S), 256, 0, st>>>(bt, g, rx, r2, sx, s2, ws.binstart, ws.chist,
                                               nullptr);

    if (ev) cudaEventRecord(ev[2], st);
    PassAArgs<T> A;
    A.g = g;
    A.bt = bt;
    A.shared = 0;
    A.nofit = nofit;
    A.px = sx;
    A.p2 = s2;
    A.binstart = ws.binstart;
    A.st = ws.stats;
    A.twA = static_cast<const Cplx<T> *>(ws.twA);
    A.tw4 = static_cast<const Cplx<T> *>(ws.tw4);
    A.H = static_cast<Cplx<T> *>(ws.H);
    {
        const void *fns[4] = {(const void *)k_passA_loop<T, false, 2>,
                              (const void *)k_passA_loop<T, true, 2>,
                              (const void *)k_passA_loop<T, false, 3>,
                              (const void *)k_passA_loop<T, true, 3>};
        for (const void *f : fns)
            if ((err = allow_max_dynamic_smem(f)) != cudaSuccess) return err;
    }
    // Pairs of adjacent column blocks write whole 32-byte sectors of each row
    // of H together (cluster store in k_passA).  Measured on the 1e6-point,
    // 1.2e7-frequency FP32 workload (2048 column blocks): pass A 0.82 ms
    // without clusters, 0.75 ms with pairs, 0.85 and 1.10 ms with clusters of
    // 4 and 8 (larger clusters wait longer at their barriers and are harder to
    // place); the small grids of batches (tens to hundreds of column blocks)
    // ran about 2% faster without.  nbins is a power of two, so cs divides it.
    int cs = g.nbins >= 512 ? 2 : 1;
    while (cs > 1 && (cs * g.BA * (int)sizeof(Cplx<T>)) % 16) cs >>= 1;
    size_t smA = passA_smem_bytes(g, sizeof(Cplx<T>), cs);
    if (cs > 1 && smA + 1024 > kSmemOptinBytes) {    // the cluster's tables do not fit
        cs = 1;
        smA = passA_smem_bytes(g, sizeof(Cplx<T>), cs);
    }
    A.cs = cs;
    // Rows of blocks: every instance gets its own row of blocks while that
    // keeps the launch within about eight blocks per SM; beyond that the blocks
    // loop over instances (tables built once per block).
    const int target = 8 * nsm;
    A.ny = 3 * S;
    // Small grids: the instances go through k_passA_group, `group` per block
    // iteration.
    const size_t cxA = sizeof(Cplx<T>);
    // a member's columns and its rows' exponent bytes
    const size_t colA = (size_t)g.BA * padded_len(g.N2) * cxA + (size_t)g.N2;
    const size_t tabA = cxA * ((size_t)g.BA * (64 + (g.N2 + 63) / 64) + 64 + (g.N2 + 63) / 64) +
                        sizeof(int) * (size_t)(g.N2 / g.fa.Rlast);
    int groupA = (int)((kGroupSmemBudget - tabA) / colA);
    groupA = groupA > 8 ? 8 : groupA;
    const int ninst = nofit ? 2 * S : 3 * S;
    // a launch whose instances all fit the two-block budget takes them in one
    // block iteration (2 blocks per SM then)
    if (ninst <= 8 && groupA < ninst && (size_t)ninst * colA + tabA <= 100 * 1024) groupA = ninst;
    // (one series' 3 transforms are grouped only when the grid has a column
    // block per SM: on narrower grids 3 rows of blocks give the launch the width
    // it lacks, measured 18 vs 37 us for pass A of a 1.8e4-cell grid, while 256
    // column blocks of FP64 ran 17% faster grouped)
    const bool grouped = cs == 1 && g.BA >= 2 && groupA >= 2 && ninst >= 2 &&
                         (ninst > 3 || g.nbins >= nsm);
    if (grouped) A.ny = 0;
    int gyA = (target + g.nbins - 1) / g.nbins;
    if (gyA < 3) gyA = 3;
    if (gyA > A.ny) gyA = A.ny;
    if (A.ny > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g.nbins, gyA);
        cfg.blockDim = dim3(kThreadsA);
        cfg.dynamicSmemBytes = smA;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const bool loop = gyA < A.ny;
        const bool three = blocks_per_sm(smA) >= 3;
        ++nk;
        if (!loop)
            err = launch_passA_single<T>(cfg, cs, A);
        else if (three)
            err = cs > 1 ? cudaLaunchKernelEx(&cfg, k_passA_loop<T, true, 3>, A)
                         : cudaLaunchKernelEx(&cfg, k_passA_loop<T, false, 3>, A);
        else
            err = cs > 1 ? cudaLaunchKernelEx(&cfg, k_passA_loop<T, true, 2>, A)
                         : cudaLaunchKernelEx(&cfg, k_passA_loop<T, false, 2>, A);
        if (err != cudaSuccess) return err;
    }
    if (grouped) {
        A.ny = 3 * S;
        A.group = groupA;
        const size_t smS = (size_t)groupA * colA + tabA;
        if ((err = allow_max_dynamic_smem((const void *)k_passA_group<T>)) != cudaSuccess)
            return err;
        int gyS = (ninst + groupA - 1) / groupA;
        const int gcap = (target + g.nbins - 1) / g.nbins;
        if (gyS > gcap) gyS = gcap;
        k_passA_group<T><<<dim3(g.nbins, gyS), kThreadsA, smS, st>>>(A);
        ++nk;
    }

    if (ev) cudaEventRecord(ev[3], st);
    PassBArgs<T> B;
    B.g = g;
    B.bt = bt;
    B.shared = 0;
    B.twB = static_cast<const Cplx<T> *>(ws.twB);
    B.H = static_cast<Cplx<T> *>(ws.H);
    B.deconv = static_cast<const T *>(ws.deconv_slot);
    B.st = ws.stats;
    B.power = power;
    B.sums = sums;
    B.nofit = nofit;
    B.norm = mode & kModeNormMask;
    // The sums carry an absolute error of about eps (sum w^ = 1), plus FP32
    // rounding on the FP32 path: an eigenvalue of M within ten times that of
    // zero is indistinguishable from a rank-deficient M (the oracle's exact
    // arithmetic uses 1e-15).
    B.lam_tol = 10.0 * fmax(g.eps, sizeof(T) == 4 ? 1e-7 : 1e-16);
    const size_t smB = passB_smem_bytes(g, sizeof(Cplx<T>));
    {
        const void *fns[6] = {(const void *)k_passB<T, 0, 2>, (const void *)k_passB<T, 1, 2>,
                              (const void *)k_passB<T, 0, 3>, (const void *)k_passB<T, 1, 3>,
                              (const void *)k_passB<T, 0, 2, kThreadsBWide>,
                              (const void *)k_passB<T, 0, 1, kThreadsBF64>};
        for (const void *f : fns)
            if ((err = allow_max_dynamic_smem(f)) != cudaSuccess) return err;
    }
    const bool threeB = blocks_per_sm(smB) >= 3;
    B.nser = S;
    int gyB = (target + g.N2 - 1) / g.N2;
    if (gyB < 1) gyB = 1;
    if (gyB > S) gyB = S;
    {
        B.stage = 0;
        // Small rows: `group` series per block iteration (power output only).
        const int nr = nofit ? 2 : 3;
        const int GB = passB_group_indep(g, sizeof(Cplx<T>), nr);
        if (GB >= 2 && S >= 2 && power && !sums) {
            if ((err = allow_max_dynamic_smem((const void *)k_passB_group<T>)) != cudaSuccess)
                return err;
            B.group = GB;
            int gy2 = (S + GB - 1) / GB;
            if (gy2 > gyB) gy2 = gyB;
            k_passB_group<T><<<dim3(g.N2, gy2), kThreadsB,
                               passB_group_smem_bytes(g, sizeof(Cplx<T>), GB, nr), st>>>(B);
        } else {
            if (threeB) k_passB<T, 0, 3><<<dim3(g.N2, gyB), kThreadsB, smB, st>>>(B);
            else if (sizeof(T) == 4)
                k_passB<T, 0, 2, kThreadsBWide><<<dim3(g.N2, gyB), kThreadsBWide, smB, st>>>(B);
            else if (kThreadsBF64 > kThreadsB && blocks_per_sm(smB) < 2)
                k_passB<T, 0, 1, kThreadsBF64><<<dim3(g.N2, gyB), kThreadsBF64, smB, st>>>(B);
            else k_passB<T, 0, 2><<<dim3(g.N2, gyB), kThreadsB, smB, st>>>(B);
        }
    }
    ++nk;
    if (ev) cudaEventRecord(ev[4], st);
    err = cudaGetLastError();
    if (err == cudaSuccess) g_pipeline_kernels.fetch_add(nk, std::memory_order_relaxed);
    return err;
}

// Shared memory of k_passA_sh for G members: their columns and row exponent
// bytes, the column tables, the root and slot tables.
static size_t passA_sh_smem_bytes(const Geometry &g, size_t cx, int G)
{
    const size_t nhi = (size_t)(g.N2 + 63) / 64;
    return (size_t)G * ((size_t)g.BA * padded_len(g.N2) * cx + (size_t)g.N2) +
           cx * ((size_t)g.BA * (64 + nhi) + 64 + nhi) + sizeof(int) * (size_t)(g.N2 / g.fa.Rlast);
}

// Shared-times batch of bt.S series (one time array t and one dy, series s's
// data at Y + y_off of its descriptor, all of nd points): the common weights,
// records, sort and w^ transforms once; per series its sums and scalars; then
// the series grids in chunks of shared_chunk_series() series, pass A and pass
// B of a chunk back to back (its grids in slots 2 .. of H, reused by every
// chunk).  ws: H of 2 + chunk grids, the common record
// sets for nd points, one series' bin tables, perm, wts, cvals (S x nd), and
// Stats / tickets for S + 1 entries (the common entry at S).
template <typename T>
cudaError_t launch_shared_pipeline(const Geometry &g, const Workspace &ws, const Batch &bt,
                                   int64_t nd, const double *t, const double *Y,
                                   const double *dy, double *power, int nred, cudaStream_t st,
                                   int mode)
{
    int nk = 0;
    cudaError_t err;
    const int nofit = (mode & kModeNoFit) ? 1 : 0;
    const int center = (!nofit || !(mode & kModeNoCenter)) ? 1 : 0;
    const int S = bt.S;
    const size_t cx = sizeof(Cplx<T>);
    int nsm = 0, dev_id = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_id);
    if (nsm <= 0) nsm = 152;
    Stats *stc = ws.stats + S;
    PointSet<T> rx = carve<T>(ws.pts_raw[0], nd), r2 = carve<T>(ws.pts_raw[1], nd);
    PointSet<T> sx = carve<T>(ws.pts_sorted[0], nd), s2 = carve<T>(ws.pts_sorted[1], nd);
    T *cvals = static_cast<T *>(ws.cvals);
    // the common records as a one-series batch
    Batch bc;
    bc.S = 1;
    bc.many = nullptr;
    bc.one = bt.one;
    bc.one.pt_off = 0;
    bc.one.y_off = 0;
    bc.one.rec_off = 0;
    bc.one.nd = nd;
    int nredc = (int)((nd + 255) / 256);
    if (nredc > 8 * nsm) nredc = 8 * nsm;
    k_sh_weights<<<nredc, 256, 0, st>>>(t, dy, nd, ws.wts, ws.partials, ws.counter + 2 * S, stc,
                                        ws.status);
    k_sh_points<T><<<nredc, 256, 0, st>>>(t, nd, bc.one.ph, g, ws.wts, rx, r2, stc);
    nk += 2;
    {
        const size_t smR = sizeof(unsigned short) * 2 * (kThreadsPts / 32) * (size_t)g.nbins;
        if ((err = allow_max_dynamic_smem((const void *)k_rank)) != cudaSuccess) return err;
        int64_t nrk = (nd + kChunk - 1) / kChunk;
        if (nrk > 8 * (int64_t)nsm) nrk = 8 * (int64_t)nsm;
        k_rank<<<dim3((unsigned)nrk, 1), kThreadsPts, smR, st>>>(bc, g, rx.ab, r2.ab, rx.rank,
                                                               ws.chist);
        k_chunk_scan<<<dim3((2 * g.nbins + 31) / 32, 1), 256, 0, st>>>(bc, g.nbins, ws.chist,
                                                                       ws.hist);
        k_scan<<<1, 1024, 0, st>>>(ws.hist, g.nbins, ws.binstart);
        int nsc = (int)((nd + 255) / 256);
        if (nsc > 4096) nsc = 4096;
        k_scatter<T><<<dim3(nsc, 1), 256, 0, st>>>(bc, g, rx, r2, sx, s2, ws.binstart, ws.chist,
                                                   ws.perm);
        nk += 4;
    }
    k_sh_stats<<<dim3(nred, S), 256, 0, st>>>(Y, bt, ws.wts, stc, ws.partials, ws.counter,
                                              ws.stats, ws.status, center);
    k_sh_series<T><<<dim3(nred, S), 256, 0, st>>>(Y, bt, ws.wts, ws.perm, sx.s[1], cvals,
                                                  ws.partials, ws.counter, ws.stats, ws.status);
    nk += 2;

    // the common w^ transforms at f and 2f (H slots 0 and 1; slot 0 is not
    // needed without a fitted mean), stage 1 of pass B deconvolves them in place
    PassAArgs<T> A;
    A.g = g;
    A.bt = bc;
    A.shared = 1;
    A.nofit = nofit;
    A.px = sx;
    A.p2 = s2;
    A.binstart = ws.binstart;
    A.st = stc;
    A.twA = static_cast<const Cplx<T> *>(ws.twA);
    A.tw4 = static_cast<const Cplx<T> *>(ws.tw4);
    A.H = static_cast<Cplx<T> *>(ws.H);
    A.ny = 2;
    A.group = 1;
    A.cv = nullptr;
    A.cstride = 0;
    {
        int cs = g.nbins >= 512 ? 2 : 1;
        while (cs > 1 && (cs * g.BA * (int)cx) % 16) cs >>= 1;
        size_t smA = passA_smem_bytes(g, cx, cs);
        if (cs > 1 && smA + 1024 > kSmemOptinBytes) {
            cs = 1;
            smA = passA_smem_bytes(g, cx, cs);
        }
        A.cs = cs;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g.nbins, 2);
        cfg.dynamicSmemBytes = smA;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if ((err = launch_passA_single<T>(cfg, cs, A)) != cudaSuccess) return err;
        ++nk;
    }
    PassBArgs<T> B;
    B.g = g;
    B.bt = bc;
    B.shared = 1;
    B.stage = 1;
    B.twB = static_cast<const Cplx<T> *>(ws.twB);
    B.H = static_cast<Cplx<T> *>(ws.H);
    B.deconv = static_cast<const T *>(ws.deconv_slot);
    B.st = stc;
    B.power = power;
    B.sums = nullptr;
    B.nofit = nofit;
    B.norm = mode & kModeNormMask;
    B.lam_tol = 10.0 * fmax(g.eps, sizeof(T) == 4 ? 1e-7 : 1e-16);
    B.nser = 1;
    B.group = 1;
    {
        const size_t smB = passB_smem_bytes(g, cx);
        if ((err = allow_max_dynamic_smem((const void *)k_passB<T, 1, 2>)) != cudaSuccess ||
            (err = allow_max_dynamic_smem((const void *)k_passB<T, 1, 3>)) != cudaSuccess)
            return err;
        if (blocks_per_sm(smB) >= 3) k_passB<T, 1, 3><<<dim3(g.N2, 1), kThreadsB, smB, st>>>(B);
        else k_passB<T, 1, 2><<<dim3(g.N2, 1), kThreadsB, smB, st>>>(B);
        ++nk;
    }

    // the series grids, chunk by chunk through H
    const size_t colA = (size_t)g.BA * padded_len(g.N2) * cx + (size_t)g.N2;
    const size_t tabA = passA_sh_smem_bytes(g, cx, 0);
    int GA = tabA + colA <= kGroupSmemBudget ? (int)((kGroupSmemBudget - tabA) / colA) : 1;
    if (GA > kMaxGroup) GA = kMaxGroup;
    const size_t smS = passA_sh_smem_bytes(g, cx, GA);
    if ((err = allow_max_dynamic_smem((const void *)k_passA_sh<T, 8>)) != cudaSuccess ||
        (err = allow_max_dynamic_smem((const void *)k_passA_sh<T, 16>)) != cudaSuccess)
        return err;
    if ((err = allow_max_dynamic_smem((const void *)k_passB_series<T>)) != cudaSuccess) return err;
    const int GB = passB_group(g, cx);
    const size_t smBS = passB_series_smem_bytes(g, cx, GB);
    const int64_t C = shared_chunk_series(g.n, cx, S);
    const int target = 8 * nsm;
    for (int64_t c0 = 0; c0 < S; c0 += C) {
        const int Sc = (int)(S - c0 < C ? S - c0 : C);
        Batch bk;
        bk.S = Sc;
        bk.many = bt.many ? bt.many + c0 : nullptr;
        bk.one = bt.one;
        PassAArgs<T> Ak = A;
        Ak.bt = bk;
        Ak.st = ws.stats + c0;
        Ak.ny = Sc;
        Ak.group = GA;
        Ak.cs = 1;
        Ak.cv = cvals + (size_t)c0 * (size_t)nd;
        Ak.cstride = nd;
        int gyA = (Sc + GA - 1) / GA;
        const int capA = (target + g.nbins - 1) / g.nbins;
        if (gyA > capA) gyA = capA;
        if (g.BA <= 8) k_passA_sh<T, 8><<<dim3(g.nbins, gyA), kThreadsA, smS, st>>>(Ak);
        else k_passA_sh<T, 16><<<dim3(g.nbins, gyA), kThreadsA, smS, st>>>(Ak);
        PassBArgs<T> Bk = B;
        Bk.bt = bk;
        Bk.st = ws.stats + c0;
        Bk.stage = 2;
        Bk.nser = Sc;
        Bk.group = GB;
        int gyB = (Sc + GB - 1) / GB;
        const int capB = (target + g.N2 - 1) / g.N2;
        if (gyB > capB) gyB = capB;
        if (gyB < 1) gyB = 1;
        k_passB_series<T><<<dim3(g.N2, gyB), kThreadsB, smBS, st>>>(Bk);
        nk += 2;
    }
    err = cudaGetLastError();
    if (err == cudaSuccess) g_pipeline_kernels.fetch_add(nk, std::memory_order_relaxed);
    return err;
}

template <typename T>
cudaError_t launch_deconv_table(const Geometry &g, void *deconv, int64_t count,
                                const double *gl_z, const double *gl_wpsi, int q,
                                cudaStream_t st)
{
    int nb = (int)((count + 255) / 256);
    if (nb > 65535) nb = 65535;
    k_deconv<T><<<nb, 256, 0, st>>>(static_cast<T *>(deconv), count, (double)g.w / (double)g.n,
                                     (double)g.w, gl_z, gl_wpsi, q);
    return cudaGetLastError();
}

template cudaError_t launch_pipeline<float>(const Geometry &, const Workspace &, int64_t,
                                            const Batch &, int64_t, const double *,
                                            const double *, const double *, double *, double *,
                                            int, cudaStream_t, cudaEvent_t *, int);
template cudaError_t launch_pipeline<double>(const Geometry &, const Workspace &, int64_t,
                                             const Batch &, int64_t, const double *,
                                             const double *, const double *, double *, double *,
                                             int, cudaStream_t, cudaEvent_t *, int);
template cudaError_t launch_shared_pipeline<float>(const Geometry &, const Workspace &,
                                                   const Batch &, int64_t, const double *,
                                                   const double *, const double *, double *, int,
                                                   cudaStream_t, int);
template cudaError_t launch_shared_pipeline<double>(const Geometry &, const Workspace &,
                                                    const Batch &, int64_t, const double *,
                                                    const double *, const double *, double *, int,
                                                    cudaStream_t, int);
// Self-test support: ff_to_double against the FP64 conversions and add on n
// pairs (hi, lo), lo within half an ulp of hi, drawn from a counter-based
// generator (splitmix64 of seed + i): general values over every exponent and
// both signs, powers of two (the binade-crossing branch), exponents next to
// the fast path's lower bound, ties at the double's rounding position, zero,
// subnormal and non-finite hi.  Counts the pairs whose bits differ.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__global__ void k_ff_assembly_check(long long n, unsigned long long seed, unsigned long long *bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long r = splitmix64(seed + (unsigned long long)i);
        const unsigned long long r2 = splitmix64(r);
        const unsigned sign = (unsigned)(r >> 63) << 31;
        unsigned e = 1u + (unsigned)((r >> 40) % 254u);          // biased exponent of hi
        unsigned mant = (unsigned)(r & 0x7FFFFFu);
        const int kind = (int)(i & 7);
        if (kind == 5) mant = 0u;                                    // a power of two
        if (kind == 6) e = 49u + (unsigned)((r >> 40) % 8u);         // around 2^-75
        if (kind == 4 && (r2 & 3u) == 0u) e = (r2 & 4u) ? 255u : 0u; // non-finite / zero, subnormal
        const float hi = __uint_as_float(sign | (e << 23) | mant);
        float lo;
        if (kind == 7 && e >= 80u && e < 255u) {
            // (k + 1/2) units of the double's ulp 2^(e - 179): a tie, |k| < 2^22
            const int k = (int)((r2 >> 8) & 0x3FFFFFu) - (1 << 21);
            lo = ((float)k + 0.5f) * __uint_as_float((e - 52u) << 23);
        } else {
            // u in [-1, 1) times ulp(hi) / 2 = 2^(e - 151) (exact scaling)
            const float u = (float)(int)(r2 >> 40) * 0x1p-23f - 1.0f;
            const float half_ulp = e >= 25u ? __uint_as_float((e - 24u) << 23)   // 2^(e - 151)
                                            : ldexpf(1.0f, (int)e - 151);
            lo = (e == 0u || e == 255u) ? u * 0x1p-149f : u * half_ulp;
        }
        const double a = ff_to_double(ff{hi, lo});
        const double b = (double)hi + (double)lo;
        if (__double_as_longlong(a) != __double_as_longlong(b) && !(a != a && b != b))
            atomicAdd(bad, 1ull);
    }
}

cudaError_t launch_ff_assembly_check(long long n, unsigned long long seed, unsigned long long *bad,
                                     cudaStream_t st)
{
    int nb = (int)((n + 255) / 256);
    if (nb > 4096) nb = 4096;
    k_ff_assembly_check<<<nb, 256, 0, st>>>(n, seed, bad);
    return cudaGetLastError();
}

cudaError_t launch_kernel_eval_pair(int n, double beta, double *dfl_out, double *fp64_out,
                                    cudaStream_t st)
{
    k_kernel_eval_pair<<<(n + 255) / 256, 256, 0, st>>>(n, beta, dfl_out, fp64_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deconv_slot(const Geometry &g, void *out, const void *compact, int64_t count,
                               cudaStream_t st)
{
    int64_t nb = (g.n + 255) / 256;
    if (nb > 8192) nb = 8192;
    k_deconv_slot<T><<<(int)nb, 256, 0, st>>>(static_cast<T *>(out),
                                               static_cast<const T *>(compact), count, g);
    return cudaGetLastError();
}

template cudaError_t launch_deconv_slot<float>(const Geometry &, void *, const void *, int64_t,
                                               cudaStream_t);
template cudaError_t launch_deconv_slot<double>(const Geometry &, void *, const void *, int64_t,
                                                cudaStream_t);
template cudaError_t launch_deconv_table<float>(const Geometry &, void *, int64_t, const double *,
                                                const double *, int, cudaStream_t);
template cudaError_t launch_deconv_table<double>(const Geometry &, void *, int64_t, const double *,
                                                 const double *, int, cudaStream_t);
template size_t point_record_bytes<float>();
template size_t point_record_bytes<double>();

}  // namespace nls
