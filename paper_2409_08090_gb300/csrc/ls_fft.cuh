// Shared-memory mixed-radix FFT used by both passes of the four-step
// fine-grid transform (the "FFT" step of the NUFFT in Sec. 1 of arXiv
// 2409.08090).  Sign convention: X[k] = sum_m x[m] exp(+2 pi i k m / L), the
// sign of the type-1 transform (Eq. 2), so Re g = C and Im g = S.
//
// Each transform runs in place as a decimation-in-frequency (Gentleman-Sande)
// sequence of radix-R stages, R in {2, 3, 4, 5, 8}: the output is left in
// digit-reversed order and read back through digit_rev().  Every butterfly
// reads and writes the same R slots, so one buffer suffices and a stage needs
// only a barrier at its end.
#pragma once

#include "ls_internal.cuh"

namespace nls {

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk2(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk2(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// (+i) * a
template <typename V> __device__ __forceinline__ V mul_i(V a) { return mk2(-a.y, a.x); }
template <typename V, typename T> __device__ __forceinline__ V cscale(V a, T s) { return mk2(a.x * s, a.y * s); }

// R-point DFT with the + sign, in registers.
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

// exp(+2 pi i p / L) from the two-level root table of length L.
template <typename V>
__device__ __forceinline__ V root(const V *twlo, const V *twhi, int p) {
    return cmul(twlo[p & (kTwSplit - 1)], twhi[p >> 6]);
}

// One DIF stage of radix R on `ncol` transforms of length L (stride colstride
// between transforms), current sub-transform length Ls.
template <int R, typename V>
__device__ __forceinline__ void dif_stage(V *buf, int ncol, int colstride, int L, int Ls,
                                          const V *twlo, const V *twhi)
{
    const int m = Ls / R;
    const int nb = L / R;
    const int tmul = L / Ls;
    const int total = ncol * nb;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int col = e / nb;
        const int bi = e - col * nb;
        const int q = bi / m;
        const int j = bi - q * m;
        V *p = buf + col * colstride + q * Ls + j;
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * m];
        Dft<R>::run(v);
        if (j != 0) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = cmul(v[k], root(twlo, twhi, j * k * tmul));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * m] = v[r];
    }
}

// In-place DIF FFT of `ncol` transforms of length rd.L held in shared memory.
// Ends with a barrier; output in digit-reversed order.
template <typename V>
__device__ void fft_dif(V *buf, int ncol, int colstride, const Radices &rd, const V *twlo,
                        const V *twhi)
{
    int Ls = rd.L;
    for (int s = 0; s < rd.count; ++s) {
        const int R = rd.rad[s];
        switch (R) {
        case 8: dif_stage<8>(buf, ncol, colstride, rd.L, Ls, twlo, twhi); break;
        case 5: dif_stage<5>(buf, ncol, colstride, rd.L, Ls, twlo, twhi); break;
        case 4: dif_stage<4>(buf, ncol, colstride, rd.L, Ls, twlo, twhi); break;
        case 3: dif_stage<3>(buf, ncol, colstride, rd.L, Ls, twlo, twhi); break;
        default: dif_stage<2>(buf, ncol, colstride, rd.L, Ls, twlo, twhi); break;
        }
        Ls /= R;
        __syncthreads();
    }
}

// Slot of output k after fft_dif: the first stage's digit (k mod R_0) selects
// the block of length L/R_0, and so on down the stages.
__device__ __forceinline__ int digit_rev(int k, const Radices &rd)
{
    int pos = 0, m = rd.L;
    for (int s = 0; s < rd.count; ++s) {
        const int R = rd.rad[s];
        m /= R;
        const int q = k / R;
        pos += (k - q * R) * m;
        k = q;
    }
    return pos;
}

}  // namespace nls
