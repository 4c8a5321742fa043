// Internal declarations shared by the host code and the kernels of the
// Lomb-Scargle NUFFT library (method of arXiv 2409.08090, Sec. 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nifty_ls.h"

namespace nls {

constexpr int kMaxStages = 8;     // stages of one sub-FFT
constexpr int kTw4Bits = 12;      // four-step twiddle table split: W^p = lo[p % 4096] * hi[p / 4096]
constexpr int kThreadsA = 256;
// Single-instance pass-A blocks of the FP32 path: 12 warps (two blocks per SM,
// 80 registers; on the 1.9e7-cell grid 0.68 ms against 0.72 ms with 8 warps).
constexpr int kThreadsAWide = 384;
// FP64 path (one block per SM on the large grids): threads of the single-
// instance pass-A block and of the pass-B block where only one fits an SM
// (1.9e7-cell grid: pass A 4.17 ms with 256 threads, 5.12 ms with 512; pass B
// 3.36 ms with 256, 3.28 ms with 512 or 768).
constexpr int kThreadsAF64 = 256;
constexpr int kThreadsBF64 = 512;
constexpr size_t kSmemOptinBytes = 232448;   // opt-in shared memory per block (227 KB)
constexpr int kThreadsB = 256;
// Pass-B blocks of the FP32 path where shared memory holds two blocks per SM:
// 12 warps each (the row transforms deal their butterflies to all of them).
constexpr int kThreadsBWide = 384;
// Column strides of pass A's per-column four-step twiddle tables (low part: 64
// entries, high part: nhi): padded so that a warp of the cluster store, whose
// lanes read columns 0 .. 3 of the cluster at one or two entries each, spreads
// the columns over the banks (a stride of 4 mod 8 entries of 8 bytes puts
// neighbouring columns 8 banks apart) instead of stacking them in one bank.
constexpr int kAloStride = 68;
__host__ __device__ constexpr int ahi_stride(int nhi) { return nhi + ((4 - nhi) & 7); }
constexpr int kMinN1 = 32;        // keeps every kernel footprint (w <= 16) within two columns

// Device status word bits (sticky until ls_sync).
// Model/normalisation word of the execute calls (the `norm` argument of the
// C-ABI): bits 0-7 the normalisation (0 standard, 1 model, 2 log, 3 psd),
// kModeNoFit: no offset in the model (C = S = 0, the w^ transform at f is not
// taken), kModeNoCenter: with kModeNoFit, y is not centred.
constexpr int kModeNormMask = 0xFF;
constexpr int kModeNoFit = 0x100;
constexpr int kModeNoCenter = 0x200;
constexpr int kStatBadInput = 1;
constexpr int kStatDegenerate = 2;

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

// One in-place DIF stage: sub-transforms of length Ls = R * m; butterfly
// (q, j) touches slots q*Ls + j + r*m, r < R.  nb = L / R butterflies.
struct FftStage {
    int R, Ls, m, nb;
    int shift;      // log2(m) if m is a power of two, else -1
    float inv_m;    // 1/m and 1/nb for small exact divisions
    float inv_nb;
    int lin;        // 1: slot of element base + r*m is pad16(base) + off[r] for every butterfly
    int off[16];
};

struct FftPlan {
    int L;
    int nstages;
    int Rlast;      // radix of the last stage (a power of two)
    int logRlast;
    FftStage st[kMaxStages];
};

// The fine grid and its four-step split: n = N1 * N2, cell m = a + N1 * b.
// Pass A takes length-N2 transforms over b (one per column a), pass B
// length-N1 transforms over a (one per row d).
struct Geometry {
    int64_t n;
    int N1, N2;
    int BA;        // columns per pass-A block (power of two)
    int logBA;
    int nbins;     // N1 / BA
    int w;
    double beta;
    double eps;    // tolerance the tables were built for
    FftPlan fa;    // length N2
    FftPlan fb;    // length N1
};

// Point records, one set per spread geometry (x and 2x).  `ab` packs the
// first covered cell c0 = a + N1 b as a | (b << 16); `roff` is such that the
// kernel argument of cell c0 + i is z = (roff - w/2 + i) * 2/w.  `rank` (the
// unsorted set of geometry x only) holds each record's stable rank among the
// records of its chunk that share its bin, geometry x in the low and 2x in
// the high 16 bits.
template <typename T> struct PointSet {
    uint32_t *ab;
    T *roff;
    typename Cx<T>::type *s[2];   // strengths (geometry x: s1, s2; geometry 2x: s3)
    uint32_t *rank;
};

// Stable bin sort: records are ranked in chunks of kChunk consecutive input
// records (one block of kThreadsPts threads, each warp kChunk / 8 of them);
// series s of a launch owns the chunk rows chunk_row0(s) .. of the chunk
// histogram, so rows never overlap: (rec_off + nd) / kChunk - rec_off / kChunk
// + 1 >= ceil(nd / kChunk).
constexpr int kChunk = 4096;
constexpr int kThreadsPts = 256;
__host__ __device__ inline int64_t chunk_row0(int64_t rec_off, int s) { return rec_off / kChunk + s; }
// Chunk-histogram entries a launch of S series over `points` records needs.
__host__ __device__ inline int64_t chunk_hist_entries(int64_t points, int S, int nbins)
{
    return (points / kChunk + S) * 2 * (int64_t)nbins;
}

// FP64 reductions are summed per fixed chunk of kRedChunk consecutive points
// (a block of 256 threads in a fixed order), and the chunk partials in a fixed
// tree, so a series' sums do not depend on how many blocks or series a launch
// has.  Series s of a launch owns the partial rows red_row0(rec_off, s) .. (3
// doubles each); a launch of S series over `points` records needs
// red_rows(points, S) rows.
constexpr int kRedChunk = 2048;
__host__ __device__ inline int64_t red_row0(int64_t rec_off, int s) { return rec_off / kRedChunk + s; }
__host__ __device__ inline int64_t red_rows(int64_t points, int64_t S) { return points / kRedChunk + S + 1; }

struct Stats {            // FP64 reductions, in device memory
    double W;             // sum of w_j
    double WY;            // sum of w_j y_j
    double WY2;           // sum of w_j y_j^2
    double ybar;          // weighted mean
    double invW;
    double scale;         // ~1/std(y): strengths are formed from scale * (y - ybar)
    double YY;            // sum of w^_j (scale (y_j - ybar))^2, the power's denominator
    double Y2;            // sum of w^_j y_j^2 (scale for the degeneracy test)
    unsigned smax[3];     // per transform (s1, s2, s3): bits of an FP32 upper bound of the
                          // largest strength component magnitude (the FP64 spread's grid)
    // set with YY, for pass B: the psd factor W YY / (2 scale^2), 1 / scale, and
    // YY as a double-float pair (one evaluation per series instead of one FP64
    // division per thread of every pass-B block)
    double psd;
    double unscale;
    float yy_hi, yy_lo;
};

struct Workspace {
    void *H;              // 3 grids of n complex T, layout [grid][d][a]
    void *pts_raw[2];     // unsorted point records (two geometries), see PointSet
    void *pts_sorted[2];
    int *hist;            // 2 * nbins records per bin, per series
    int *binstart;        // 2 * (nbins + 1), per series
    int *chist;           // chunk histograms, then their prefixes over chunks:
                          // rows of 2 * nbins (chunk_row0, chunk_hist_entries)
    double *partials;     // reduction partials: 3 doubles per row (red_rows)
    unsigned int *counter;// last-block tickets (2)
    Stats *stats;
    int *status;          // device status word
    void *twA;            // two-level root table for length N2: lo (64) then hi (ceil(N2/64))
    void *twB;            // two-level root table for length N1
    void *tw4;            // four-step table for n: lo (4096) then hi (ceil(n/4096))
    void *deconv;         // 1/phi_hat(k'), k' = 0 .. K0max
    void *deconv_slot;    // the same in pass-B order: [d * N1 + slot], n entries
    // shared-times batches (launch_shared_pipeline)
    int *perm;            // common sorted order -> input index (geometry x)
    double *wts;          // common weights 1/dy^2
    void *cvals;          // per series, c_i = scale (y - ybar) in the sorted order
};

// Series grids per pass-A/pass-B round of a shared-times batch: a chunk's fine
// grids (kSharedChunkBytes) are written by pass A and read back by pass B, and
// the next chunk reuses their slots of H.  Measured on 4096 series of 1.8e5
// cells (FP32): chunks of 48 MB (L2-resident between the passes) 28.0 ms per
// batch, 192 MB 24.7 ms, one chunk 21.1 ms: the passes are not HBM-bound, and
// every chunk adds the launches' tails and per-block set-up, so chunks only
// bound the workspace.
constexpr int64_t kSharedChunkBytes = 4ll << 30;

inline int64_t shared_chunk_series(int64_t n, size_t cx, int64_t S)
{
    int64_t c = kSharedChunkBytes / (n * (int64_t)cx);
    if (c < 1) c = 1;
    return c < S ? c : S;
}

// Frequencies of one series, decomposed for the exact phase reduction:
// df = df_m 2^df_e, f0 = (-1)^f0_neg f0_m 2^f0_e, centre mode K0.
struct PhaseArgs {
    uint64_t df_m, f0_m;
    int df_e, f0_e, f0_neg;
    int64_t K0;
};

// One series of a launch: its points [pt_off, pt_off + nd) of t, y, dy, its
// point records [rec_off, rec_off + nd) of the workspace, its nf outputs at
// power[out_off ...] (sums at 6 out_off).
struct SeriesDesc {
    int64_t pt_off, y_off, rec_off, nd;   // t, dy at pt_off; y at y_off
    int64_t out_off, nf;
    PhaseArgs ph;
};

// S series launched together (grid dimension y): `many` points to S device
// descriptors, or is null and the single series is `one`.  Per-series
// workspace: stats[s], counter[2s .. 2s+1], partials[s * 3 * nred ...],
// hist[s * 2 * nbins ...], binstart[s * 2 * (nbins + 1) ...], chist from row
// chunk_row0(rec_off, s),
// H[s * 3 * n ...].
struct Batch {
    int S;
    SeriesDesc one;
    const SeriesDesc *many;
};

// x = +-m 2^e with m < 2^53, the exact decomposition of a finite double.
void decompose_double(double x, uint64_t &m, int &e, int &neg);

// `ev`, if not null, holds LS_NUM_STAGES + 1 events recorded at the stage
// boundaries.  `capacity` = points the record arrays hold; `max_nd` = largest
// series of the batch; nred = reduction blocks per series.
// Pipeline kernels enqueued (or recorded into graphs) by this process.
long long pipeline_kernel_count();

template <typename T>
cudaError_t launch_pipeline(const Geometry &g, const Workspace &ws, int64_t capacity,
                            const Batch &b, int64_t max_nd, const double *t, const double *y,
                            const double *dy, double *power, double *sums, int nred,
                            cudaStream_t st, cudaEvent_t *ev, int mode = 0);

// Shared-times batch (one time array and one dy for all bt.S series): see
// the definition.  Stats and tickets hold S + 1 entries.
template <typename T>
cudaError_t launch_shared_pipeline(const Geometry &g, const Workspace &ws, const Batch &bt,
                                   int64_t nd, const double *t, const double *Y,
                                   const double *dy, double *power, int nred, cudaStream_t st,
                                   int mode);

template <typename T>
cudaError_t launch_deconv_table(const Geometry &g, void *deconv, int64_t count,
                                const double *gl_z, const double *gl_wpsi, int q,
                                cudaStream_t st);

// Reorder the deconvolution table into pass-B order: entry d * N1 + pos holds
// 1/phi_hat of the mode min(k, n - k), k = d + N2 * (frequency of slot pos),
// or 0 past the table's `count` entries (modes no grid of the plan needs).
template <typename T>
cudaError_t launch_deconv_slot(const Geometry &g, void *out, const void *compact, int64_t count,
                               cudaStream_t st);

// Self-test: the FP64 path's double-float kernel evaluation and the FP64 one
// at n points of [-1, 1] (device buffers of n doubles each).
// Self-test: the FP32 path's integer-pipe double assembly against the FP64
// conversions and add on n generated pairs; *bad (device) counts mismatches.
cudaError_t launch_ff_assembly_check(long long n, unsigned long long seed, unsigned long long *bad,
                                     cudaStream_t st);

cudaError_t launch_kernel_eval_pair(int n, double beta, double *dfl_out, double *fp64_out,
                                    cudaStream_t st);

template <typename T>
size_t point_record_bytes();

// Stage descriptors of a length-L sub-FFT with radices up to maxr (false if L
// has no schedule).
bool fft_plan_for_length(int L, FftPlan *fp, int maxr);

// The planned path's automatic tile width (columns per pass-A block) and the
// largest FFT radix of pass A (length n2) and pass B (length n1).
void plan_tiling(int prec, int n1, int n2, int *ba, int *maxrA, int *maxrB);

// Quadrature rule of the deconvolution table for kernel width w and shape
// beta: nodes z in [0, 1] and weights times psi(z); returns the node count, or
// -1 (nothing written) when it exceeds cap.
int es_quadrature_into(int w, double beta, double *z, double *wpsi, int cap);

size_t passA_smem_bytes(const Geometry &g, size_t cx_bytes, int cs);
size_t passB_smem_bytes(const Geometry &g, size_t cx_bytes);

}  // namespace nls
