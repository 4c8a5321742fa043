// Shared-memory mixed-radix FFT used by both passes of the four-step
// fine-grid transform (the "FFT" step of the NUFFT in Sec. 1 of arXiv
// 2409.08090).  Sign convention: X[k] = sum_m x[m] exp(+2 pi i k m / L), the
// sign of the type-1 transform (Eq. 2), so Re g = C and Im g = S.
//
// Each transform runs in place as a decimation-in-frequency (Gentleman-Sande)
// sequence of radix-R stages, R in {18, 9, 3, 5} first and then {16, 8, 4, 2},
// each butterfly an R-point DFT in registers.  Every butterfly reads and writes the
// same R slots, so one buffer suffices and a stage needs only a barrier at its
// end.  The output is left in digit-reversed order; slot_to_freq() gives the
// frequency index each slot holds.  Twiddles exp(2 pi i j k / Ls) =
// W_L^(j k L/Ls) come from a two-level root table of W_L = exp(2 pi i / L) held
// in shared memory (W_L^p = lo[p % 64] * hi[p / 64], both exactly rounded from
// FP64), so a stage's twiddles never leave the SM.
#pragma once

#include "ls_internal.cuh"

namespace nls {

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

// Double-float numbers for the transforms of the FP64 path: a value is
// hi + lo with two FP32 parts (about 48 significant bits), so the FFT runs on
// the FP32 units (this part issues FP64 at 1/64 of the FP32 rate).  Sum:
// Knuth's two-sum of the high parts with the low parts added in, an error
// below 2^-47 (|a| + |b|), so transform errors stay bounded by the input norm
// as with FP64; product: the fma two-product.  Spreading, deconvolution and
// the power stay in FP64.
struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};
struct alignas(16) dfl2 {
    dfl x, y;
};
__device__ __forceinline__ dfl operator+(dfl a, dfl b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return dfl(h, e - (h - s));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const float h = p + e;
    return dfl(h, e - (h - p));
}
__device__ __forceinline__ dfl2 mk2(dfl a, dfl b)
{
    dfl2 r;
    r.x = a;
    r.y = b;
    return r;
}

// Complex type the transforms run in, per storage precision, and conversions.
template <typename T> struct FftOf;
template <> struct FftOf<float> { using type = float2; };
template <> struct FftOf<double> { using type = dfl2; };
__device__ __forceinline__ float2 to_fft(float2 v) { return v; }
__device__ __forceinline__ dfl2 to_fft(double2 v) { return mk2(dfl(v.x), dfl(v.y)); }
__device__ __forceinline__ float2 from_fft(float2 v) { return v; }
// hi + lo rounded to the nearest double, from the bit patterns on the integer
// pipe (for |lo| <= ulp(hi) / 2, as double-float values are kept; others take
// the FP64 path below):
// hi widens exactly (exponent rebiased, mantissa shifted up 29 bits) and lo,
// in units of that double's ulp 2^(e - 52) (e the unbiased exponent of hi,
// |lo| <= 2^28 units), is rounded to an integer (ties to even, the rounding of
// the FP64 add) and added to the bits.  The sum stays in hi's binade except
// where hi is a power of two and lo points towards zero, and for hi zero,
// subnormal, non-finite or below 2^-75: those take the FP64 conversions and
// add (same value), out of line so that the common path does not issue them
// predicated.  This part converts and adds FP64 at 1/64 of the FP32 rate.
__device__ __noinline__ double hl_to_double_fp64(float hi, float lo)
{
    return (double)hi + (double)lo;
}
__device__ __forceinline__ double hl_to_double(float hi, float lo)
{
    const unsigned hb = __float_as_uint(hi);
    const unsigned e = (hb >> 23) & 0xffu;
    if (e < 52u || e == 255u || (hb & 0x7fffffu) == 0u) return hl_to_double_fp64(hi, lo);
    const float units = __uint_as_float((306u - e) << 23);          // 2^(52 - (e - 127))
    int r = __float2int_rn(lo * units);
    if (r > (1 << 28) || r < -(1 << 28)) return hl_to_double_fp64(hi, lo);   // |lo| > ulp(hi)/2
    if (hb >> 31) r = -r;
    const unsigned long long mag = ((unsigned long long)(hb & 0x7fffffffu) + (896ull << 23)) << 29;
    return __longlong_as_double((long long)(((unsigned long long)(hb >> 31) << 63) |
                                            (mag + (unsigned long long)(long long)r)));
}
__device__ __forceinline__ double2 from_fft(dfl2 v)
{
    return make_double2(hl_to_double(v.x.hi, v.x.lo), hl_to_double(v.y.hi, v.y.lo));
}

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk2(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk2(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// (+i) * a and (-i) * a
template <typename V> __device__ __forceinline__ V mul_i(V a) { return mk2(-a.y, a.x); }
template <typename V> __device__ __forceinline__ V mul_mi(V a) { return mk2(a.y, -a.x); }
template <typename V, typename T> __device__ __forceinline__ V cscale(V a, T s) { return mk2(a.x * s, a.y * s); }

// R-point DFT with the + sign, in registers, natural order in and out.
template <int R> struct Dft;

template <> struct Dft<2> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        V a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};

template <> struct Dft<3> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        using T = decltype(v[0].x);
        const T h = T(0.86602540378443864676);  // sin(2 pi / 3)
        V t1 = cadd(v[1], v[2]);
        V t2 = csub(v[0], cscale(t1, T(0.5)));
        V t3 = cscale(csub(v[1], v[2]), h);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, mul_i(t3));
        v[2] = csub(t2, mul_i(t3));
    }
};

template <> struct Dft<4> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        V c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, mul_i(d));
        v[3] = csub(b, mul_i(d));
    }
};

template <> struct Dft<5> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        using T = decltype(v[0].x);
        const T c1 = T(0.30901699437494742410);   // cos(2 pi / 5)
        const T c2 = T(-0.80901699437494742410);  // cos(4 pi / 5)
        const T s1 = T(0.95105651629515357212);   // sin(2 pi / 5)
        const T s2 = T(0.58778525229247312917);   // sin(4 pi / 5)
        V x0 = v[0];
        V a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
        V b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
        V p1 = mk2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
        V p2 = mk2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
        V q1 = mk2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
        V q2 = mk2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
        v[0] = cadd(x0, cadd(a1, a2));
        v[1] = cadd(p1, mul_i(q1));
        v[4] = csub(p1, mul_i(q1));
        v[2] = cadd(p2, mul_i(q2));
        v[3] = csub(p2, mul_i(q2));
    }
};

template <> struct Dft<8> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        using T = decltype(v[0].x);
        const T r = T(0.70710678118654752440);  // 1/sqrt(2)
        V e[4] = {v[0], v[2], v[4], v[6]};
        V o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4>::run(e);
        Dft<4>::run(o);
        // o[k] *= exp(+2 pi i k / 8)
        o[1] = mk2((o[1].x - o[1].y) * r, (o[1].x + o[1].y) * r);
        o[2] = mul_i(o[2]);
        o[3] = mk2(-(o[3].x + o[3].y) * r, (o[3].x - o[3].y) * r);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};

// 9 = 3 x 3: x index n = 3 n1 + n2, output k = k1 + 3 k2 (one stage where two
// radix-3 stages would each read and write the whole transform).
template <> struct Dft<9> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        using T = decltype(v[0].x);
        const V w1 = mk2(T(0.76604444311897803520), T(0.64278760968653932632));   // e^{2 pi i / 9}
        const V w2 = mk2(T(0.17364817766693034885), T(0.98480775301220805936));   // e^{4 pi i / 9}
        const V w4 = mk2(T(-0.93969262078590838405), T(0.34202014332566873304));  // e^{8 pi i / 9}
        V y[3][3];
#pragma unroll
        for (int n2 = 0; n2 < 3; ++n2) {
            V a[3] = {v[n2], v[n2 + 3], v[n2 + 6]};
            Dft<3>::run(a);
#pragma unroll
            for (int k1 = 0; k1 < 3; ++k1) y[n2][k1] = a[k1];
        }
        // y[n2][k1] *= exp(+2 pi i n2 k1 / 9)
        y[1][1] = cmul(y[1][1], w1);
        y[1][2] = cmul(y[1][2], w2);
        y[2][1] = cmul(y[2][1], w2);
        y[2][2] = cmul(y[2][2], w4);
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            V b[3] = {y[0][k1], y[1][k1], y[2][k1]};
            Dft<3>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) v[k1 + 3 * k2] = b[k2];
        }
    }
};

// 18 = 2 x 9: x index n = 9 n1 + n2, output k = k1 + 2 k2: radix-2 butterflies
// over n1, the twiddles exp(+2 pi i n2 k1 / 18), two 9-point DFTs over n2 (one
// stage where a radix-9 and a radix-2 stage would each read and write the
// whole transform).
template <> struct Dft<18> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        using T = decltype(v[0].x);
        const T c20 = T(0.93969262078590838405), s20 = T(0.34202014332566873304);
        const T c40 = T(0.76604444311897803520), s40 = T(0.64278760968653932632);
        const T c80 = T(0.17364817766693034885), s80 = T(0.98480775301220805936);
        const T s60 = T(0.86602540378443864676);
        V a[9], b[9];
#pragma unroll
        for (int n2 = 0; n2 < 9; ++n2) {
            a[n2] = cadd(v[n2], v[n2 + 9]);
            b[n2] = csub(v[n2], v[n2 + 9]);
        }
        b[1] = cmul(b[1], mk2(c20, s20));
        b[2] = cmul(b[2], mk2(c40, s40));
        b[3] = cmul(b[3], mk2(T(0.5), s60));
        b[4] = cmul(b[4], mk2(c80, s80));
        b[5] = cmul(b[5], mk2(-c80, s80));
        b[6] = cmul(b[6], mk2(T(-0.5), s60));
        b[7] = cmul(b[7], mk2(-c40, s40));
        b[8] = cmul(b[8], mk2(-c20, s20));
        Dft<9>::run(a);
        Dft<9>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) {
            v[2 * k2] = a[k2];
            v[2 * k2 + 1] = b[k2];
        }
    }
};

// 16 = 4 x 4: x index n = 4 n1 + n2, output k = k1 + 4 k2.
template <> struct Dft<16> {
    template <typename V> __device__ __forceinline__ static void run(V *v) {
        using T = decltype(v[0].x);
        const T c = T(0.92387953251128675613);   // cos(pi / 8)
        const T s = T(0.38268343236508977173);   // sin(pi / 8)
        const T r = T(0.70710678118654752440);   // cos(pi / 4)
        V y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            V a[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
            Dft<4>::run(a);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = a[k1];
        }
        // y[n2][k1] *= exp(+2 pi i n2 k1 / 16)
        y[1][1] = cmul(y[1][1], mk2(c, s));
        y[1][2] = mk2((y[1][2].x - y[1][2].y) * r, (y[1][2].x + y[1][2].y) * r);
        y[1][3] = cmul(y[1][3], mk2(s, c));
        y[2][1] = mk2((y[2][1].x - y[2][1].y) * r, (y[2][1].x + y[2][1].y) * r);
        y[2][2] = mul_i(y[2][2]);
        y[2][3] = mk2(-(y[2][3].x + y[2][3].y) * r, (y[2][3].x - y[2][3].y) * r);
        y[3][1] = cmul(y[3][1], mk2(s, c));
        y[3][2] = mk2(-(y[3][2].x + y[3][2].y) * r, (y[3][2].x - y[3][2].y) * r);
        y[3][3] = cmul(y[3][3], mk2(-c, -s));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            V b[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Dft<4>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
        }
    }
};

__device__ __host__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__device__ __host__ __forceinline__ int padded_len(int L) { return L + (L >> 4) + 1; }

// floor(a / b) for 0 <= a < 2^22 by a float reciprocal and one correction.
__device__ __forceinline__ int small_div(int a, int b, float inv_b)
{
    int q = __float2int_rz((float)a * inv_b);
    const int r = a - q * b;
    if (r < 0) --q;
    else if (r >= b) ++q;
    return q;
}

// exp(2 pi i p / L) from the two-level root table (lo: 64 entries, hi: L/64).
template <typename V>
__device__ __forceinline__ V root_tw(const V *roots, int p)
{
    return cmul(roots[p & 63], roots[64 + (p >> 6)]);
}

// The twiddles W_L^(k step), k = 1 .. R-1, of one butterfly.  FP32: from two
// table lookups, W^step and W^(4 step): with k = 4a + b, W^(k step) is
// W^(4a step) W^(b step), and each factor is a power of its looked-up root
// formed by at most two products, so every twiddle is within a few rounded
// products of the table; fifteen lookups of the table's two levels per
// radix-16 butterfly become two, with as many complex products as before.
// Double-float: one lookup per twiddle (the six double-float powers held at
// once cost the 80-register kernels spills).
template <int R, typename V>
struct Twiddles {
    static constexpr bool kPow = sizeof(V) == 8;
    static constexpr int kA = (R - 1) / 4;   // largest a
    V wb[4];                                 // W^(b step), b = 1 .. 3
    V wa[kA + 1];                            // W^(4 a step), a = 1 .. kA
    const V *roots;
    int step;
    __device__ __forceinline__ Twiddles(const V *roots_, int step_) : roots(roots_), step(step_)
    {
        if constexpr (kPow) {
            wb[1] = root_tw(roots, step);
            if constexpr (R > 2) wb[2] = cmul(wb[1], wb[1]);
            if constexpr (R > 3) wb[3] = cmul(wb[2], wb[1]);
            if constexpr (kA >= 1) wa[1] = root_tw(roots, 4 * step);
            if constexpr (kA >= 2) wa[2] = cmul(wa[1], wa[1]);
            if constexpr (kA >= 3) wa[3] = cmul(wa[2], wa[1]);
            if constexpr (kA >= 4) wa[4] = cmul(wa[2], wa[2]);
            static_assert(kA <= 4, "radix above 20");
        }
    }
    // k is a constant after unrolling
    __device__ __forceinline__ V get(int k) const
    {
        if constexpr (!kPow) return root_tw(roots, k * step);
        const int a = k >> 2, b = k & 3;
        if (a == 0) return wb[b];
        if (b == 0) return wa[a];
        return cmul(wa[a], wb[b]);
    }
};

// Load the two-level root table of length L into shared memory in the
// transform's type (no barrier).
template <typename W, typename V>
__device__ __forceinline__ void load_roots(W *dst, const V *__restrict__ src, int L)
{
    const int cnt = 64 + ((L + 63) >> 6);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[i] = to_fft(__ldg(src + i));
}

// Frequency index held by output slot pos of fft_dif: pos = sum_s d_s m_s
// with m_s = L / (R_0 ... R_s); the index is sum_s d_s R_0 ... R_{s-1}.
__device__ __forceinline__ int slot_to_freq(int pos, const FftPlan &fp)
{
    int c = 0, mult = 1;
    for (int s = 0; s < fp.nstages; ++s) {
        const FftStage &st = fp.st[s];
        int dgt;
        if (st.shift >= 0) {
            dgt = pos >> st.shift;
        } else {
            dgt = small_div(pos, st.m, st.inv_m);
        }
        pos -= dgt * st.m;
        c += dgt * mult;
        mult *= st.R;
    }
    return c;
}

// Frequency index of slot pos with the per-block table D[i] =
// slot_to_freq(i * Rlast): the last stage's digit is pos mod Rlast and
// contributes (pos mod Rlast) * L / Rlast.
__device__ __forceinline__ int slot_freq_tab(int pos, const int *D, const FftPlan &fp)
{
    return D[pos >> fp.logRlast] + (pos & (fp.Rlast - 1)) * (fp.L >> fp.logRlast);
}

// Fill D (L / Rlast entries) in shared memory (no barrier).
__device__ __forceinline__ void fill_slot_table(int *D, const FftPlan &fp)
{
    const int cnt = fp.L >> fp.logRlast;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) D[i] = slot_to_freq(i << fp.logRlast, fp);
}

// Butterfly bi of one DIF stage of radix R over NC transforms (stride
// colstride) processed together: the NC groups of loads are in flight at once
// and each twiddle is formed once.
template <int R, int NC, typename V>
__device__ __forceinline__ void dif_butterfly(V *buf, int colstride, const FftStage &st,
                                              const V *roots, int tmul, int bi)
{
    const int m = st.m;
    int q, j;
    if (st.shift >= 0) {
        q = bi >> st.shift;
        j = bi & (m - 1);
    } else {
        q = small_div(bi, m, st.inv_m);
        j = bi - q * m;
    }
    const int base = q * st.Ls + j;
    const int pb = pad16(base);
    int off[R];
#pragma unroll
    for (int r = 0; r < R; ++r) off[r] = st.lin ? pb + st.off[r] : pad16(base + r * m);
    V v[NC][R];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[c][r] = buf[c * colstride + off[r]];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) Dft<R>::run(v[c]);
    if (j != 0) {
        const Twiddles<R, V> tw(roots, j * tmul);   // W_Ls^(j k) = W_L^(k j tmul)
#pragma unroll
        for (int k = 1; k < R; ++k) {
            const V w = tw.get(k);
#pragma unroll
            for (int c = 0; c < NC; ++c) v[c][k] = cmul(v[c][k], w);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[c * colstride + off[r]] = v[c][r];
    }
}

// One DIF stage of radix R over NC transforms: a thread takes butterfly (q, j)
// of every transform.
template <int R, int NC, typename V>
__device__ __forceinline__ void dif_stage(V *buf, int colstride, const FftStage &st,
                                          const V *roots, int L)
{
    const int tmul = L / st.Ls;
    for (int bi = threadIdx.x; bi < st.nb; bi += blockDim.x)
        dif_butterfly<R, NC>(buf, colstride, st, roots, tmul, bi);
}

// One DIF stage over ncol transforms with the (transform, butterfly) pairs
// dealt to the block's threads in turn, one transform per thread at a time:
// for blocks with more threads than a stage has butterflies per transform.
template <int R, typename V>
__device__ __forceinline__ void dif_stage_dealt(V *buf, int ncol, int colstride,
                                                const FftStage &st, const V *roots, int L)
{
    const int tmul = L / st.Ls;
    const int nb = st.nb;
    const float inv_nb = 1.0f / (float)nb;
    for (int u = threadIdx.x; u < ncol * nb; u += blockDim.x) {
        const int c = small_div(u, nb, inv_nb);
        dif_butterfly<R, 1>(buf + c * colstride, colstride, st, roots, tmul, u - c * nb);
    }
}

// The first stage over columns that still hold the spread's fixed-point pairs
// (FP32 path): element i of column c is the int pair at slot pad16(i), in
// units of 2^(e - 30) with e = rexp of its row (rows of column c: rexp +
// (c / BA) * rstride), or zero without a load where e marks an empty row.
// The stage converts while it loads and writes FP32 complex values back to the
// same slots (same bytes per cell), so no separate conversion pass is needed.
constexpr signed char kEmptyRow = -128;
template <int R, int NC>
__device__ __forceinline__ void dif_stage_first_fixed(float2 *buf, int colstride, const FftStage &st,
                                                      const float2 *roots, int L,
                                                      const signed char *rexp, int BA, int rstride,
                                                      int c0)
{
    const int m = st.m;
    const int tmul = L / st.Ls;
    const int2 *ibuf = reinterpret_cast<const int2 *>(buf);
    for (int bi = threadIdx.x; bi < st.nb; bi += blockDim.x) {
        int q, j;
        if (st.shift >= 0) {
            q = bi >> st.shift;
            j = bi & (m - 1);
        } else {
            q = small_div(bi, m, st.inv_m);
            j = bi - q * m;
        }
        const int base = q * st.Ls + j;
        const int pb = pad16(base);
        int off[R];
#pragma unroll
        for (int r = 0; r < R; ++r) off[r] = st.lin ? pb + st.off[r] : pad16(base + r * m);
        float2 v[NC][R];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const signed char *re = rexp + ((c0 + c) / BA) * rstride;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = re[base + r * m];
                if (e == kEmptyRow) {
                    v[c][r] = make_float2(0.f, 0.f);
                } else {
                    const int2 iv = ibuf[c * colstride + off[r]];
                    const float unit = __int_as_float((127 - 30 + e) << 23);
                    v[c][r] = make_float2(__int2float_rn(iv.x) * unit, __int2float_rn(iv.y) * unit);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) Dft<R>::run(v[c]);
        if (j != 0) {
            const Twiddles<R, float2> tw(roots, j * tmul);
#pragma unroll
            for (int k = 1; k < R; ++k) {
                const float2 w = tw.get(k);
#pragma unroll
                for (int c = 0; c < NC; ++c) v[c][k] = cmul(v[c][k], w);
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[c * colstride + off[r]] = v[c][r];
        }
    }
}

template <int R, int G>
__device__ __forceinline__ void first_stage_fixed_cols(float2 *buf, int ncol, int colstride,
                                                       const FftStage &st, const float2 *roots,
                                                       int L, const signed char *rexp, int BA,
                                                       int rstride)
{
    int c0 = 0;
    if (G > 1) {
        for (; c0 + G <= ncol; c0 += G)
            dif_stage_first_fixed<R, G>(buf + c0 * colstride, colstride, st, roots, L, rexp, BA,
                                        rstride, c0);
    }
    for (; c0 < ncol; ++c0)
        dif_stage_first_fixed<R, 1>(buf + c0 * colstride, colstride, st, roots, L, rexp, BA,
                                    rstride, c0);
}

// One stage over `ncol` transforms, G at a time (G = 1 for the remainder).
template <int R, int G, typename V>
__device__ __forceinline__ void dif_stage_cols(V *buf, int ncol, int colstride, const FftStage &st,
                                               const V *roots, int L)
{
    int c0 = 0;
    if (G > 1) {
        for (; c0 + G <= ncol; c0 += G) dif_stage<R, G>(buf + c0 * colstride, colstride, st, roots, L);
    }
    for (; c0 < ncol; ++c0) dif_stage<R, 1>(buf + c0 * colstride, colstride, st, roots, L);
}

// In-place DIF FFT of `ncol` transforms of length fp.L in shared memory
// (padded layout, columns colstride apart), up to NC of them per thread at a
// time, NC16 for radix 16 (at most 2 by default, to stay within 128 registers
// in FP32; 1 for blocks compiled for 80).  Ends with a barrier; output in
// digit-reversed order (see slot_to_freq).
template <int NC, int NC16 = (NC < 2 ? NC : 2), typename V>
__device__ void fft_dif(V *buf, int ncol, int colstride, const FftPlan &fp, const V *roots,
                        int first = 0)
{
    for (int s = first; s < fp.nstages; ++s) {
        const FftStage &st = fp.st[s];
        switch (st.R) {
        case 18: dif_stage_cols<18, 1>(buf, ncol, colstride, st, roots, fp.L); break;
        case 16: dif_stage_cols<16, NC16>(buf, ncol, colstride, st, roots, fp.L); break;
        case 9: dif_stage_cols<9, NC>(buf, ncol, colstride, st, roots, fp.L); break;
        case 8: dif_stage_cols<8, NC>(buf, ncol, colstride, st, roots, fp.L); break;
        case 4: dif_stage_cols<4, NC>(buf, ncol, colstride, st, roots, fp.L); break;
        case 5: dif_stage_cols<5, NC>(buf, ncol, colstride, st, roots, fp.L); break;
        case 3: dif_stage_cols<3, NC>(buf, ncol, colstride, st, roots, fp.L); break;
        default: dif_stage_cols<2, NC>(buf, ncol, colstride, st, roots, fp.L); break;
        }
        __syncthreads();
    }
}

// In-place DIF FFT of `ncol` transforms of length fp.L with every stage's
// (transform, butterfly) pairs dealt to all threads (dif_stage_dealt).  Ends
// with a barrier; output in digit-reversed order.
template <typename V>
__device__ void fft_dif_dealt(V *buf, int ncol, int colstride, const FftPlan &fp, const V *roots)
{
    for (int s = 0; s < fp.nstages; ++s) {
        const FftStage &st = fp.st[s];
        switch (st.R) {
        case 18: dif_stage_dealt<18>(buf, ncol, colstride, st, roots, fp.L); break;
        case 16: dif_stage_dealt<16>(buf, ncol, colstride, st, roots, fp.L); break;
        case 9: dif_stage_dealt<9>(buf, ncol, colstride, st, roots, fp.L); break;
        case 8: dif_stage_dealt<8>(buf, ncol, colstride, st, roots, fp.L); break;
        case 4: dif_stage_dealt<4>(buf, ncol, colstride, st, roots, fp.L); break;
        case 5: dif_stage_dealt<5>(buf, ncol, colstride, st, roots, fp.L); break;
        case 3: dif_stage_dealt<3>(buf, ncol, colstride, st, roots, fp.L); break;
        default: dif_stage_dealt<2>(buf, ncol, colstride, st, roots, fp.L); break;
        }
        __syncthreads();
    }
}

// fft_dif over FP32 columns holding the spread's fixed-point pairs: the
// first stage converts as it loads (dif_stage_first_fixed), the rest run as
// usual.  Ends with a barrier.
template <int NC, int NC16 = (NC < 2 ? NC : 2)>
__device__ void fft_dif_fixed(float2 *buf, int ncol, int colstride, const FftPlan &fp,
                              const float2 *roots, const signed char *rexp, int BA, int rstride)
{
    const FftStage &st = fp.st[0];
    switch (st.R) {
    case 18: first_stage_fixed_cols<18, 1>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    case 16: first_stage_fixed_cols<16, NC16>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    case 9: first_stage_fixed_cols<9, NC>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    case 8: first_stage_fixed_cols<8, NC>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    case 4: first_stage_fixed_cols<4, NC>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    case 5: first_stage_fixed_cols<5, NC>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    case 3: first_stage_fixed_cols<3, NC>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    default: first_stage_fixed_cols<2, NC>(buf, ncol, colstride, st, roots, fp.L, rexp, BA, rstride); break;
    }
    __syncthreads();
    fft_dif<NC, NC16>(buf, ncol, colstride, fp, roots, 1);
}

}  // namespace nls
