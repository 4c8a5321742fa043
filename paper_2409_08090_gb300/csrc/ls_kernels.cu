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
#include <math.h>

#include "ls_fft.cuh"
#include "ls_internal.cuh"

namespace nls {

template <typename T> using Cplx = typename Cx<T>::type;

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

// ---------------------------------------------------------------------------
// K1a: weights and weighted mean (FP64).  W = sum 1/dy^2, WY = sum y/dy^2.
// ---------------------------------------------------------------------------
__global__ void k_stats(const double *__restrict__ t, const double *__restrict__ y,
                        const double *__restrict__ dy, int64_t nd, double *partials,
                        unsigned int *counter, Stats *st, int *status)
{
    __shared__ double sh[32];
    double sw = 0.0, swy = 0.0;
    int bad = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nd;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double d = dy ? dy[j] : 1.0;
        const double yj = y[j];
        const double w = 1.0 / (d * d);
        bad |= !(d > 0.0) || !isfinite(d) || !isfinite(yj) || !isfinite(t[j]) || !isfinite(w);
        sw += w;
        swy += w * yj;
    }
    if (bad) atomicOr(status, kStatBadInput);
    double a = block_sum(sw, sh);
    double b = block_sum(swy, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
    if (last_block(counter)) {
        if (threadIdx.x == 0) {
            double W = 0.0, WY = 0.0;
            for (unsigned int i = 0; i < gridDim.x; ++i) {
                W += __ldcg(partials + 2 * i);
                WY += __ldcg(partials + 2 * i + 1);
            }
            st->W = W;
            st->WY = WY;
            st->ybar = WY / W;
            *counter = 0u;
        }
    }
}

// Split a fine-grid position u in [0, n] (cells) into the first covered cell
// c0 = ceil(u - w/2) (wrapped into [0, n)) and roff = c0 - u + w/2 in [0, 1].
__device__ __forceinline__ void split_cell(double u, int64_t n, int w, int &c0, double &roff)
{
    const double lo = ceil(u - 0.5 * w);
    roff = lo - u + 0.5 * w;
    int64_t c = (int64_t)lo;
    if (c < 0) c += n;
    if (c >= n) c -= n;
    c0 = (int)c;
}

// frac(a * t) for a double-double a = a_hi + a_lo, accurate to ~1e-16 cycles
// whatever the size of a t (error-free product of a_hi t by fma).
__device__ __forceinline__ double frac_dd(double a_hi, double a_lo, double t)
{
    const double p = a_hi * t;
    const double e = fma(a_hi, t, -p);
    double r = (p - floor(p)) + (e + a_lo * t);
    return r - floor(r);
}

// exp(2 pi i c) for a cycle count c in [0, 1) (FP64 phase).
template <typename T> __device__ __forceinline__ void cis_cycles(double c, double &re, double &im);

template <> __device__ __forceinline__ void cis_cycles<double>(double c, double &re, double &im)
{
    sincospi(2.0 * c, &im, &re);
}

// FP32 path: the reduced phase is split as c = cf + dc (cf the nearest float);
// sincospif(2 cf) is corrected to first order in 2 pi dc (|dc| < 3e-8, so the
// neglected term is < 1e-14).  The result is rounded to FP32 by the caller.
template <> __device__ __forceinline__ void cis_cycles<float>(double c, double &re, double &im)
{
    const double cr = c - rint(c);
    const float cf = (float)cr;
    const double dc = 6.283185307179586477 * (cr - (double)cf);
    float sf, cfv;
    sincospif(2.0f * cf, &sf, &cfv);
    re = (double)cfv - dc * (double)sf;
    im = (double)sf + dc * (double)cfv;
}

// ---------------------------------------------------------------------------
// K1b: per-point records (FP64 arithmetic, stored in T) + bin histogram +
// YY reduction.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_points(const double *__restrict__ t, const double *__restrict__ y,
                         const double *__restrict__ dy, int64_t nd, double df, double fc_hi,
                         double fc_lo, Geometry g, PointSet<T> px, PointSet<T> p2, int *hist,
                         double *partials, unsigned int *counter, Stats *st, int *status)
{
    __shared__ double sh[32];
    const double W = st->W;
    const double ybar = st->ybar;
    const double n_d = (double)g.n;
    double syy = 0.0, sy2 = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nd;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double tj = t[j], yj = y[j];
        const double d = dy ? dy[j] : 1.0;
        const double wh = 1.0 / (d * d * W);
        const double yc = yj - ybar;
        syy += wh * yc * yc;
        sy2 += wh * yj * yj;
        // NUFFT coordinates in cycles: frac(df t) and frac(2 df t), exact product.
        const double ph = frac_dd(df, 0.0, tj);
        double ph2 = 2.0 * ph;
        ph2 -= floor(ph2);
        int c1, c2;
        double r1, r2;
        split_cell(ph * n_d, g.n, g.w, c1, r1);
        split_cell(ph2 * n_d, g.n, g.w, c2, r2);
        // Pre-phase p = exp(2 pi i fc t) and p^2.
        const double pc = frac_dd(fc_hi, fc_lo, tj);
        double pc2 = 2.0 * pc;
        pc2 -= floor(pc2);
        double pr, pi, qr, qi;
        cis_cycles<T>(pc, pr, pi);
        cis_cycles<T>(pc2, qr, qi);
        const double a = wh * yc;
        px.cell[j] = c1;
        px.roff[j] = (T)r1;
        px.s[0][j] = mk2((T)(a * pr), (T)(a * pi));
        px.s[1][j] = mk2((T)(wh * pr), (T)(wh * pi));
        p2.cell[j] = c2;
        p2.roff[j] = (T)r2;
        p2.s[0][j] = mk2((T)(wh * qr), (T)(wh * qi));
        atomicAdd(&hist[(c1 % g.N1) / g.BA], 1);
        atomicAdd(&hist[g.nbins + (c2 % g.N1) / g.BA], 1);
    }
    double a = block_sum(syy, sh);
    double b = block_sum(sy2, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
    if (last_block(counter)) {
        if (threadIdx.x == 0) {
            double YY = 0.0, Y2 = 0.0;
            for (unsigned int i = 0; i < gridDim.x; ++i) {
                YY += __ldcg(partials + 2 * i);
                Y2 += __ldcg(partials + 2 * i + 1);
            }
            st->YY = YY;
            st->Y2 = Y2;
            // A constant series: variance zero up to the rounding of the mean.
            if (!(YY > 1e-24 * Y2)) atomicOr(status, kStatDegenerate);
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// K2: exclusive scan of the two histograms (one block) -> bin starts, cursors.
// ---------------------------------------------------------------------------
__global__ void k_scan(const int *__restrict__ hist, int nbins, int *binstart, int *cursor)
{
    __shared__ int chunk_tot[1024];
    for (int geo = 0; geo < 2; ++geo) {
        const int *h = hist + geo * nbins;
        int *bs = binstart + geo * (nbins + 1);
        int *cu = cursor + geo * nbins;
        const int per = (nbins + blockDim.x - 1) / blockDim.x;
        const int lo = threadIdx.x * per;
        const int hi = min(nbins, lo + per);
        int s = 0;
        for (int i = lo; i < hi; ++i) s += h[i];
        chunk_tot[threadIdx.x] = s;
        __syncthreads();
        // inclusive scan of chunk totals (Hillis-Steele)
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            int v = (threadIdx.x >= (unsigned)off) ? chunk_tot[threadIdx.x - off] : 0;
            __syncthreads();
            chunk_tot[threadIdx.x] += v;
            __syncthreads();
        }
        int run = (threadIdx.x == 0) ? 0 : chunk_tot[threadIdx.x - 1];
        for (int i = lo; i < hi; ++i) {
            bs[i] = run;
            cu[i] = run;
            run += h[i];
        }
        if (threadIdx.x == blockDim.x - 1) bs[nbins] = chunk_tot[blockDim.x - 1];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K2b: scatter the point records into bin order (order inside a bin is free).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_scatter(int64_t nd, Geometry g, PointSet<T> rx, PointSet<T> r2,
                          PointSet<T> sx, PointSet<T> s2, int *cursor)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nd;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int c1 = rx.cell[j];
        const int d1 = atomicAdd(&cursor[(c1 % g.N1) / g.BA], 1);
        sx.cell[d1] = c1;
        sx.roff[d1] = rx.roff[j];
        sx.s[0][d1] = rx.s[0][j];
        sx.s[1][d1] = rx.s[1][j];
        const int c2 = r2.cell[j];
        const int d2 = atomicAdd(&cursor[g.nbins + (c2 % g.N1) / g.BA], 1);
        s2.cell[d2] = c2;
        s2.roff[d2] = r2.roff[j];
        s2.s[0][d2] = r2.s[0][j];
    }
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
    PointSet<T> px, p2;
    const int *binstart;   // 2 * (nbins + 1)
    const Cplx<T> *twA;    // N2 root table (lo, hi)
    const Cplx<T> *tw4;    // n four-step table (lo 4096, hi)
    Cplx<T> *H;
};

template <typename T>
__device__ __forceinline__ T es_kernel(T z, T beta)
{
    const T s = sqrt(fmax(T(0), T(1) - z * z));
    return exp(beta * (s - T(1)));
}

template <typename T>
__global__ void __launch_bounds__(kThreadsA) k_passA(PassAArgs<T> A)
{
    using V = Cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = A.g;
    const int N1 = g.N1, N2 = g.N2, BA = g.BA;
    V *buf = reinterpret_cast<V *>(smem_raw);
    V *twlo = buf + (size_t)BA * N2;
    V *twhi = twlo + kTwSplit;
    const int nhi = (N2 + kTwSplit - 1) / kTwSplit;

    const int grid = blockIdx.y;
    const int blk = blockIdx.x;
    const int a0 = blk * BA;

    for (int i = threadIdx.x; i < kTwSplit + nhi; i += blockDim.x) twlo[i] = A.twA[i];
    for (int i = threadIdx.x; i < BA * N2; i += blockDim.x) buf[i] = mk2(T(0), T(0));
    __syncthreads();

    // ---- spread ----
    const PointSet<T> &P = (grid < 2) ? A.px : A.p2;
    const V *str = (grid == 1) ? A.px.s[1] : P.s[0];
    const int *bs = A.binstart + ((grid < 2) ? 0 : (g.nbins + 1));
    const int nbb = (g.w - 1 + BA - 1) / BA;   // bins before this one that reach it
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
    const T halfw = T(0.5) * T(g.w);
    const T zscale = T(2) / T(g.w);
    const T beta = T(g.beta);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int j = (e < cnt0) ? (r0s + e) : (r1s + e - cnt0);
        const int c0 = P.cell[j];
        const T roff = P.roff[j];
        const V s = str[j];
        int aa = c0 % N1;
        int bb = c0 / N1;
        for (int i = 0; i < g.w; ++i) {
            const int ca = aa - a0;
            if (ca >= 0 && ca < BA) {
                const T z = (roff - halfw + T(i)) * zscale;
                const T v = es_kernel(z, beta);
                V *dst = buf + (size_t)ca * N2 + bb;
                atomicAdd(&dst->x, s.x * v);
                atomicAdd(&dst->y, s.y * v);
            }
            if (++aa == N1) {
                aa = 0;
                if (++bb == N2) bb = 0;
            }
        }
    }
    __syncthreads();

    // ---- column FFTs over b ----
    fft_dif(buf, BA, N2, g.radA, twlo, twhi);

    // ---- twiddle exp(2 pi i a d / n) and store H[grid][d][a] ----
    const V *t4lo = A.tw4;
    const V *t4hi = A.tw4 + (1 << kTw4Bits);
    V *H = A.H + (size_t)grid * (size_t)g.n;
    for (int e = threadIdx.x; e < BA * N2; e += blockDim.x) {
        const int c = e % BA;
        const int d = e / BA;
        const int a = a0 + c;
        V v = buf[(size_t)c * N2 + digit_rev(d, g.radA)];
        const int64_t p = (int64_t)a * d;   // < n
        const V tw = cmul(t4lo[p & ((1 << kTw4Bits) - 1)], t4hi[p >> kTw4Bits]);
        H[(size_t)d * N1 + a] = cmul(v, tw);
    }
}

// ---------------------------------------------------------------------------
// Pass B: for row d, FFT the three grids over a (length N1), deconvolve the
// needed modes and evaluate the power in FP64.
// ---------------------------------------------------------------------------
template <typename T>
struct PassBArgs {
    Geometry g;
    const Cplx<T> *twB;
    const Cplx<T> *H;
    const T *deconv;       // 1/phi_hat(|k'|)
    const Stats *st;
    int64_t nf, K0;
    double *power;
    double *sums;
};

// Generalised (floating-mean) power, standard normalisation, from the six sums
// and YY (FP64).  With CC = sum w^ cos^2 - C^2 = (1 + C2)/2 - C^2,
// SS = (1 - C2)/2 - S^2, CS = S2/2 - C S, the 2x2 system M = [[CC, CS], [CS, SS]]
// is diagonalised by the rotation through w tau (tan 2 w tau =
// (S2 - 2CS)/(C2 - (C^2 - S^2))), so YC_tau^2/CC_tau + YS_tau^2/SS_tau =
// v^T M^-1 v with v = (Ch, Sh).  The closed form needs no trigonometry; a
// nearly singular M (all phases equal mod pi) falls back to the explicit tau
// rotation, dropping a vanishing CC_tau or SS_tau term.
__device__ __forceinline__ double ls_power(double Ch, double Sh, double C, double S, double C2,
                                           double S2, double YY)
{
    const double CC = 0.5 * (1.0 + C2) - C * C;
    const double SS = 0.5 * (1.0 - C2) - S * S;
    const double CS = 0.5 * S2 - C * S;
    const double D = CC * SS - CS * CS;
    if (D > 1e-12 * (CC * CC + SS * SS) && D > 1e-30) {
        const double N = Ch * Ch * SS - 2.0 * Ch * Sh * CS + Sh * Sh * CC;
        return N / (D * YY);
    }
    // tau rotation: cos/sin of 2 w tau, then half-angle.
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
    if (CCt > 1e-15) p += YC * YC / CCt;
    if (SSt > 1e-15) p += YS * YS / SSt;
    return p / YY;
}

template <typename T>
__global__ void __launch_bounds__(kThreadsB) k_passB(PassBArgs<T> B)
{
    using V = Cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geometry &g = B.g;
    const int N1 = g.N1, N2 = g.N2;
    V *buf = reinterpret_cast<V *>(smem_raw);
    V *twlo = buf + 3 * (size_t)N1;
    V *twhi = twlo + kTwSplit;
    const int nhi = (N1 + kTwSplit - 1) / kTwSplit;
    const int d = blockIdx.x;

    for (int i = threadIdx.x; i < kTwSplit + nhi; i += blockDim.x) twlo[i] = B.twB[i];
    for (int gi = 0; gi < 3; ++gi) {
        const V *src = B.H + (size_t)gi * (size_t)g.n + (size_t)d * N1;
        for (int a = threadIdx.x; a < N1; a += blockDim.x) buf[(size_t)gi * N1 + a] = src[a];
    }
    __syncthreads();

    fft_dif(buf, 3, N1, g.radB, twlo, twhi);

    const double YY = B.st->YY;
    const int64_t n = g.n;
    const int64_t hi_start = n - B.K0;
    const int64_t lo_end = B.nf - B.K0;
    for (int c = threadIdx.x; c < N1; c += blockDim.x) {
        const int64_t k = d + (int64_t)N2 * c;
        int64_t kp;
        if (k < lo_end) kp = k;
        else if (k >= hi_start) kp = k - n;
        else continue;
        const int pos = digit_rev(c, g.radB);
        const T dc = B.deconv[kp < 0 ? -kp : kp];
        const V g1 = buf[pos], g2 = buf[N1 + pos], g3 = buf[2 * N1 + pos];
        const double Ch = (double)(g1.x * dc), Sh = (double)(g1.y * dc);
        const double C = (double)(g2.x * dc), S = (double)(g2.y * dc);
        const double C2 = (double)(g3.x * dc), S2 = (double)(g3.y * dc);
        const int64_t out = kp + B.K0;
        if (B.power) B.power[out] = ls_power(Ch, Sh, C, S, C2, S2, YY);
        if (B.sums) {
            double *o = B.sums + 6 * out;
            o[0] = Ch; o[1] = Sh; o[2] = C; o[3] = S; o[4] = C2; o[5] = S2;
        }
    }
}

// ---------------------------------------------------------------------------
// Deconvolution table: 1/phi_hat(k), phi_hat(k) = w int_0^1 psi(z) cos(pi k w z / n) dz
// by a Gauss-Legendre rule on [0, 1] (nodes z, weights already times psi(z)).
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

// ---------------------------------------------------------------------------
// Host-side launch helpers
// ---------------------------------------------------------------------------
template <typename T>
size_t point_record_bytes()
{
    return sizeof(int) + sizeof(T) + 2 * sizeof(Cplx<T>);
}

size_t passA_smem_bytes(const Geometry &g, size_t cx)
{
    return cx * ((size_t)g.BA * g.N2 + kTwSplit + (g.N2 + kTwSplit - 1) / kTwSplit);
}

size_t passB_smem_bytes(const Geometry &g, size_t cx)
{
    return cx * (3 * (size_t)g.N1 + kTwSplit + (g.N1 + kTwSplit - 1) / kTwSplit);
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
    p.cell = reinterpret_cast<int *>(b + off);
    return p;
}

template <typename T>
cudaError_t launch_pipeline(const Geometry &g, const Workspace &ws, int64_t max_nd,
                            const ExecParams &p, int nred, cudaStream_t st, cudaEvent_t *ev)
{
    cudaError_t err;
    PointSet<T> rx = carve<T>(ws.pts_raw[0], max_nd), r2 = carve<T>(ws.pts_raw[1], max_nd);
    PointSet<T> sx = carve<T>(ws.pts_sorted[0], max_nd), s2 = carve<T>(ws.pts_sorted[1], max_nd);

    if (ev) cudaEventRecord(ev[0], st);
    err = cudaMemsetAsync(ws.hist, 0, sizeof(int) * 2 * (size_t)g.nbins, st);
    if (err != cudaSuccess) return err;
    k_stats<<<nred, 256, 0, st>>>(p.t, p.y, p.dy, p.nd, ws.partials, ws.counter, ws.stats,
                                  ws.status);
    k_points<T><<<nred, 256, 0, st>>>(p.t, p.y, p.dy, p.nd, p.df, p.fc_hi, p.fc_lo, g, rx, r2,
                                      ws.hist, ws.partials, ws.counter + 1, ws.stats, ws.status);
    if (ev) cudaEventRecord(ev[1], st);
    k_scan<<<1, 1024, 0, st>>>(ws.hist, g.nbins, ws.binstart, ws.cursor);
    const int nsc = (int)((p.nd + 255) / 256 < 4096 ? (p.nd + 255) / 256 : 4096);
    k_scatter<T><<<nsc, 256, 0, st>>>(p.nd, g, rx, r2, sx, s2, ws.cursor);

    if (ev) cudaEventRecord(ev[2], st);
    PassAArgs<T> A;
    A.g = g;
    A.px = sx;
    A.p2 = s2;
    A.binstart = ws.binstart;
    A.twA = static_cast<const Cplx<T> *>(ws.twA);
    A.tw4 = static_cast<const Cplx<T> *>(ws.tw4);
    A.H = static_cast<Cplx<T> *>(ws.H);
    const size_t smA = passA_smem_bytes(g, sizeof(Cplx<T>));
    err = cudaFuncSetAttribute(k_passA<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smA);
    if (err != cudaSuccess) return err;
    k_passA<T><<<dim3(g.nbins, 3), kThreadsA, smA, st>>>(A);

    if (ev) cudaEventRecord(ev[3], st);
    PassBArgs<T> B;
    B.g = g;
    B.twB = static_cast<const Cplx<T> *>(ws.twB);
    B.H = static_cast<const Cplx<T> *>(ws.H);
    B.deconv = static_cast<const T *>(ws.deconv);
    B.st = ws.stats;
    B.nf = p.nf;
    B.K0 = p.K0;
    B.power = p.power;
    B.sums = p.sums;
    const size_t smB = passB_smem_bytes(g, sizeof(Cplx<T>));
    err = cudaFuncSetAttribute(k_passB<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smB);
    if (err != cudaSuccess) return err;
    k_passB<T><<<g.N2, kThreadsB, smB, st>>>(B);
    if (ev) cudaEventRecord(ev[4], st);
    return cudaGetLastError();
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
                                            const ExecParams &, int, cudaStream_t, cudaEvent_t *);
template cudaError_t launch_pipeline<double>(const Geometry &, const Workspace &, int64_t,
                                             const ExecParams &, int, cudaStream_t, cudaEvent_t *);
template cudaError_t launch_deconv_table<float>(const Geometry &, void *, int64_t, const double *,
                                                const double *, int, cudaStream_t);
template cudaError_t launch_deconv_table<double>(const Geometry &, void *, int64_t, const double *,
                                                 const double *, int, cudaStream_t);
template size_t point_record_bytes<float>();
template size_t point_record_bytes<double>();

}  // namespace nls
