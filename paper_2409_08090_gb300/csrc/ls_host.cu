// Host side of the Lomb-Scargle NUFFT library: plan construction (parameter
// choice from the tolerance, fine-grid size, four-step split, tables),
// workspace ownership and the C-ABI entry points declared in nifty_ls.h.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ls_internal.cuh"

using namespace nls;

// Parameters chosen for a plan (see ls_choose_params).
struct PlanParams {
    int32_t w, n1, n2;
    double beta, sigma, upsampling;
    int64_t n;
    int32_t cols = 0;     // requested columns per pass-A block (0: automatic)
    int32_t maxr = 0;     // requested largest FFT radix (0: 16)
};

struct ls_plan_s;
struct ls_batch_s;

// One grid class of a ragged batch: series whose frequency count maps to the
// same fine grid share these tables (sub-plan without workspace).
struct BatchClass {
    PlanParams pp;
    ls_plan_s *sub;
};

// Workspace of ls_execute_batch, grown on demand.
// Batch launches are spread over kBatchLanes streams, each with its own
// workspace, so the many small launches of a ragged batch (one per grid class)
// overlap on the device; the plan's stream waits for all of them.
constexpr int kBatchLanes = 4;

constexpr int kMaxBatchS = 16384;   // series per batch launch

// Workspace of one batch lane.  The per-launch buffers (fine grids, point
// records, bin totals and starts, chunk histograms) are carved for each launch
// from one arena (carve_launch); the per-series arrays are sized once for
// kMaxBatchS series.  The arena grows only when a launch needs more than it
// holds; ls_plan_reserve_batch sizes it to the plan's lane budget up front, so
// that later batch calls within the budget allocate nothing.
struct BatchWorkspace {
    void *arena = nullptr;
    int64_t arena_bytes = 0;
    unsigned int *counter = nullptr;   // 2 kMaxBatchS last-block tickets
    Stats *stats = nullptr;            // kMaxBatchS
    SeriesDesc *desc = nullptr;        // kMaxBatchS
    std::vector<void *> allocs;        // the per-series arrays
    int64_t bytes = 0;                 // arena + per-series arrays
};

// Offsets of one launch's buffers inside a lane arena (256-byte aligned).
struct LaunchCarve {
    size_t H, pts[4], hist, binstart, chist, partials, bytes;
    size_t perm = 0, wts = 0, cvals = 0;   // shared-times launches only
};

LaunchCarve carve_launch(int64_t n, int nbins, size_t cx, size_t recb, int64_t S, int64_t points,
                         int64_t grids)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    LaunchCarve c;
    size_t off = 0;
    c.H = off;
    off = al(off + cx * (size_t)n * (size_t)grids);
    const size_t rec = recb * (size_t)points + 5 * 256;   // carve() alignment of each set
    for (int i = 0; i < 4; ++i) {
        c.pts[i] = off;
        off = al(off + rec);
    }
    c.hist = off;
    off = al(off + sizeof(int) * 2 * (size_t)nbins * (size_t)S);
    c.binstart = off;
    off = al(off + sizeof(int) * 2 * ((size_t)nbins + 1) * (size_t)S);
    c.chist = off;
    off = al(off + sizeof(int) * (size_t)chunk_hist_entries(points, (int)S, nbins));
    c.partials = off;
    off = al(off + sizeof(double) * 3 * (size_t)red_rows(points, S));
    c.wts = off;
    off = al(off + sizeof(double) * (size_t)points);
    c.bytes = off;
    return c;
}

struct ls_plan_s {
    int device;
    cudaStream_t stream;
    int prec;
    int64_t max_nd;
    int64_t nf;
    double eps;
    double sigma;         // upsampling factor the plan chose
    double upsampling;    // requested upsampling (0: automatic)
    int32_t cols_req;     // requested columns per pass-A block (0: automatic)
    int32_t maxr_req;     // requested largest FFT radix (0: 16)
    int maxrA, maxrB;     // largest radix of the pass-A (N2) / pass-B (N1) FFT stages
    int nsm;
    Geometry g;
    Workspace ws;
    int nred;
    int64_t deconv_count;
    std::vector<void *> allocations;
    int64_t bytes;
    // staging for host-memory arguments (allocated on first use)
    double *stage_in;     // 3 * max_nd
    double *stage_out;    // nf
    double *stage_sums;   // 6 * nf
    // stage timing (ls_timing_enable)
    bool timing;
    std::vector<cudaEvent_t> tev;   // kTimingRing * (LS_NUM_STAGES + 1)
    int t_head, t_pending;
    double t_acc[LS_NUM_STAGES];
    int64_t t_count;
    // ls_execute_batch
    std::vector<BatchClass> classes;
    BatchWorkspace bws[kBatchLanes];
    cudaStream_t lane_stream[kBatchLanes] = {};
    cudaEvent_t lane_done[kBatchLanes] = {};
    cudaEvent_t lane_start = nullptr;
    int64_t batch_budget = 0;   // bytes for the batch workspaces (0: chosen on first use)
    std::vector<ls_batch_s *> batches;   // prepared batches not yet destroyed
};

// One launch of a prepared batch (ls_batch_prepare): everything but the
// data pointers, fixed at preparation.
struct PreparedLaunch {
    int lane;
    size_t cls;           // index into ls_batch_s::subs
    int S;
    int64_t points, max_nd;
    size_t desc_off;      // first descriptor in ls_batch_s::desc_all
    SeriesDesc one;
    int shared;
};

// A prepared batch owns its class tables, its per-lane workspaces and its
// device descriptors, so nothing a later call does to the plan's own batch
// state (class rebuilds, workspace growth) moves memory a recorded run uses.
struct ls_batch_s {
    ls_plan_s *plan = nullptr;   // null once the plan is destroyed (the handle is then inert)
    int norm = 0;
    std::vector<ls_plan_s *> subs;
    std::vector<PreparedLaunch> launches;
    BatchWorkspace bws[kBatchLanes];
    SeriesDesc *desc_all = nullptr;
    int64_t bytes = 0;
};

namespace {

constexpr int kTimingRing = 64;
constexpr int kEvPerSet = LS_NUM_STAGES + 1;

// Largest row (N1, pass B) and column (N2, pass A) lengths of the four-step
// split.  Pass B holds three rows of N1 in shared memory: 3 x 4096 FP64
// (double-float) values take 209 KB, one block per SM.  The most balanced split
// of a 1.9e7-cell FP64 grid is then 4096 x 4608 instead of 2048 x 9216, whose
// 147 KB pass-A columns also ran one block per SM: measured pass A 4.93 ->
// 3.78 ms, pass B 2.60 -> 3.35 ms.
constexpr int kN1MaxF32 = 4096, kN2MaxF32 = 25600;
constexpr int kN1MaxF64 = 4096, kN2MaxF64 = 12800;
constexpr size_t kSmemPairBudget = 100 * 1024;   // two pass-A blocks per SM

bool radix_schedule(int L, std::vector<int> &rad, int maxr = 16);

// Shared memory of a one-column pass-A block (the smallest block a split can
// use: padded column, per-column and root tables, slot table, row exponents)
// plus 2 KB of
// margin: a column length above the opt-in limit cannot launch.  Called for
// every candidate split of every series of a batch, so it only derives the
// radix schedule (not the verified stage tables).
bool passA_column_fits(int64_t N2, int prec)
{
    // the last radix of radix_schedule(N2) without building the schedule (this
    // runs for every candidate split of every series of a batch call)
    if (N2 > (1 << 20) || N2 < 2) return false;
    int x = (int)N2, nst = 0, last = 0;
    while (x % 9 == 0) { x /= 9; ++nst; last = 9; }
    while (x % 3 == 0) { x /= 3; ++nst; last = 3; }
    while (x % 5 == 0) { x /= 5; ++nst; last = 5; }
    int k = 0;
    while ((1 << k) < x) ++k;
    if ((1 << k) != x || k == 0) return false;
    if (k % 4) { ++nst; last = 1 << (k % 4); }
    if (k >= 4) { nst += k / 4; last = 16; }
    if (nst > kMaxStages) return false;
    const size_t cx = prec == LS_FP32 ? 8 : 16;
    const size_t nhi = (size_t)(N2 + 63) / 64;
    const size_t padded = (size_t)N2 + (size_t)N2 / 16 + 1;   // pad16 layout of the column
    const size_t bytes = cx * (padded + 2 * (kAloStride + ahi_stride((int)nhi))) +
                         sizeof(int) * (size_t)(N2 / last) + (size_t)N2 + 2048;   // + row exponents
    return bytes <= kSmemOptinBytes;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int ilog2_exact(int64_t x)
{
    int k = 0;
    while (((int64_t)1 << k) < x) ++k;
    return ((int64_t)1 << k) == x ? k : -1;
}

// Radix schedule of a sub-FFT of length L = c 2^k (c = 3^a 5^b, k >= 1): the
// odd radices first (3s paired into 9s), then one stage of 8, 4 or 2 for
// k mod 4, then 16s, so the last stage is a power of two (16 whenever k >= 4);
// a lone 2 merges into a leading 9 as one radix-18 stage.
// With maxr = 8 the power-of-two part is one stage of 4 or 2 for k mod 3 and
// then 8s (more stages, fewer registers per butterfly).
bool radix_schedule(int L, std::vector<int> &rad, int maxr)
{
    rad.clear();
    int x = L;
    while (x % 9 == 0) { rad.push_back(9); x /= 9; }
    while (x % 3 == 0) { rad.push_back(3); x /= 3; }
    while (x % 5 == 0) { rad.push_back(5); x /= 5; }
    int k = 0;
    while ((x >> k) > 1) ++k;
    if ((1 << k) != x || k == 0) return false;
    const int lr = maxr == 8 ? 3 : 4;
    if (k % lr) rad.push_back(1 << (k % lr));
    for (int i = 0; i < k / lr; ++i) rad.push_back(1 << lr);
    // a lone radix-2 stage beside a radix-9 one (radix-16 schedules of long
    // transforms): one radix-18 stage instead, a pass over the transform fewer
    // (N2 = 4608: 18, 16, 16; pass A 0.636 -> 0.627 ms; the small grids of
    // ragged batches measured 2% slower with it, so they keep 9 and 2)
    if (maxr != 8 && L >= 4096 && k % lr == 1 && k / lr >= 1 && rad[0] == 9) {
        rad[0] = 18;
        for (size_t i = 1; i < rad.size(); ++i)
            if (rad[i] == 2) {
                rad.erase(rad.begin() + (long)i);
                break;
            }
    }
    return (int)rad.size() <= kMaxStages;
}

// ES kernel width and shape for tolerance eps and upsampling factor sigma.
// sigma = 2: w = ceil(log10(1/eps)) + 1, beta = 2.30 w (the error falls about
// tenfold per extra cell).  Other sigma: the kernel's aliasing error decays as
// exp(-pi w sqrt(1 - 1/sigma)), so w = ceil(ln(1/eps) / (pi sqrt(1 - 1/sigma)))
// and beta = 0.976 pi (1 - 1/(2 sigma)) w (the same constant that gives 2.30 w
// at sigma = 2).  Returns false when the width would exceed 16 cells.
bool es_params(double eps, double sigma, int *w, double *beta)
{
    int ww;
    double bo;
    if (sigma == 2.0) {
        ww = (int)ceil(log10(1.0 / eps) - 1e-9) + 1;
        if (ww < 2) ww = 2;
        bo = 2.30;
        if (ww == 2) bo = 2.20;
        else if (ww == 3) bo = 2.26;
        else if (ww == 4) bo = 2.38;
    } else {
        ww = (int)ceil(log(1.0 / eps) / (M_PI * sqrt(1.0 - 1.0 / sigma)) - 1e-9);
        if (ww < 2) ww = 2;
        bo = 0.976 * M_PI * (1.0 - 0.5 / sigma);
    }
    if (ww > 16) return false;
    *w = ww;
    *beta = bo * ww;
    return true;
}

// Fine grid: the smallest n = c 2^k >= max(sigma nf, 2 w, 64), c in the odd
// 5-smooth set {1, 3, 5, 9, 15, 25, 27, 45, 75, 81, 125}, that splits as
// n = N1 * N2 with N1 = 2^k1 a power of two in [kMinN1, n1max] and
// N2 = n / N1 <= n2max even (the odd factor lives in N2); among the splits the
// most balanced one is taken.
ls_status choose_grid(int64_t nf, double sigma, int w, int prec, int64_t *n_out, int *n1_out,
                      int *n2_out)
{
    static const int odd[] = {1, 3, 5, 9, 15, 25, 27, 45, 75, 81, 125};
    const int n1max = prec == LS_FP32 ? kN1MaxF32 : kN1MaxF64;
    const int n2max = prec == LS_FP32 ? kN2MaxF32 : kN2MaxF64;
    int64_t nmin = (int64_t)ceil(sigma * (double)nf - 1e-9);
    if (nmin < 2 * w) nmin = 2 * w;
    if (nmin < 64) nmin = 64;
    // Candidates c 2^k in increasing order (the smallest untried multiple of
    // each c); the first with an admissible split is the smallest admissible n
    // (different c never give the same n).  Called for every series of a
    // batch call, so only the candidates up to the answer are split.
    const int64_t nlimit = (int64_t)n1max * n2max;
    int64_t cand[11];
    for (int i = 0; i < 11; ++i) {
        cand[i] = odd[i];
        while (cand[i] < nmin) cand[i] *= 2;
    }
    int64_t best_n = -1;
    int best_n1 = 0;
    for (;;) {
        int i = -1;
        for (int j = 0; j < 11; ++j)
            if (cand[j] <= nlimit && (i < 0 || cand[j] < cand[i])) i = j;
        if (i < 0) break;
        const int64_t n = cand[i];
        // most balanced admissible split of this n
        int pick = -1;
        double bal = 1e300;
        for (int k1 = ilog2_exact(kMinN1); ((int64_t)1 << k1) <= n1max; ++k1) {
            const int64_t N1 = (int64_t)1 << k1;
            if (n % N1) break;
            const int64_t N2 = n / N1;
            if (N2 > n2max || N2 < 2 || (N2 & 1) || !passA_column_fits(N2, prec)) continue;
            const double b = fabs(log((double)N1) - log((double)N2));
            if (b < bal) { bal = b; pick = (int)N1; }
        }
        if (pick > 0) {
            best_n = n;
            best_n1 = pick;
            break;
        }
        cand[i] *= 2;
    }
    if (best_n < 0) return LS_ERR_UNSUPPORTED;
    *n_out = best_n;
    *n1_out = best_n1;
    *n2_out = (int)(best_n / best_n1);
    return LS_OK;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_q).
void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &wt)
{
    x.assign(q, 0.0);
    wt.assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double z = cos(M_PI * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= q; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int quad_nodes(int w) { return 2 * w + 24; }

// Nodes on [0, 1] (the even integrand is folded) and weights times psi(z).
// The substitution z = sin(theta) removes the square-root endpoint behaviour of
// psi at z = 1 (sqrt(1 - z^2) = cos theta, dz = cos theta dtheta), so the
// Gauss-Legendre rule on theta in [0, pi/2] converges geometrically.
// Writes q = quad_nodes(w) nodes and weights and returns q, or returns -1 (and
// writes nothing) when q exceeds cap.
int es_quadrature_fill(int w, double beta, double *z, double *wpsi, int cap)
{
    const int q = quad_nodes(w);
    if (q > cap) return -1;
    std::vector<double> x, wt;
    gauss_legendre(q, x, wt);
    for (int i = 0; i < q; ++i) {
        const double th = 0.25 * M_PI * (x[i] + 1.0);
        const double c = cos(th);
        z[i] = sin(th);
        wpsi[i] = 0.25 * M_PI * wt[i] * c * exp(beta * (c - 1.0));
    }
    return q;
}

void es_quadrature(int w, double beta, std::vector<double> &z, std::vector<double> &wpsi)
{
    const int q = quad_nodes(w);
    z.resize(q);
    wpsi.resize(q);
    es_quadrature_fill(w, beta, z.data(), wpsi.data(), q);
}

// exp(2 pi i p / L) for p in [0, L), from an exact integer reduction.
void root_of_unity(int64_t p, int64_t L, double *re, double *im)
{
    p %= L;
    const double a = 2.0 * M_PI * ((double)p / (double)L);
    *re = cos(a);
    *im = sin(a);
}

template <typename T>
void fill_root_table(std::vector<T> &out, int64_t L, int split_bits)
{
    const int64_t lo = (int64_t)1 << split_bits;
    const int64_t hi = (L + lo - 1) / lo;
    out.resize(2 * (lo + hi));
    for (int64_t i = 0; i < lo; ++i) {
        double re, im;
        root_of_unity(i, L, &re, &im);
        out[2 * i] = (T)re;
        out[2 * i + 1] = (T)im;
    }
    for (int64_t i = 0; i < hi; ++i) {
        double re, im;
        root_of_unity((i * lo) % L, L, &re, &im);
        out[2 * (lo + i)] = (T)re;
        out[2 * (lo + i) + 1] = (T)im;
    }
}

ls_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return LS_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return LS_ERR_NOMEM;
    }
    return LS_ERR_CUDA;
}

ls_status plan_alloc(ls_plan_s *p, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return cuda_status(e);
    }
    p->allocations.push_back(*ptr);
    p->bytes += (int64_t)bytes;
    return LS_OK;
}

void plan_free(ls_plan_s *p)
{
    for (void *a : p->allocations) cudaFree(a);
    p->allocations.clear();
}

// Stage descriptors of a length-L DIF FFT (radix schedule, sub-lengths and
// the constants for exact small divisions).
bool build_fft(int L, FftPlan *fp, int maxr = 16)
{
    std::vector<int> rad;
    if (!radix_schedule(L, rad, maxr)) return false;
    fp->L = L;
    fp->nstages = (int)rad.size();
    int Ls = L;
    for (int s = 0; s < fp->nstages; ++s) {
        FftStage &st = fp->st[s];
        const int R = rad[s];
        st.R = R;
        st.Ls = Ls;
        st.m = Ls / R;
        st.nb = L / R;
        st.shift = ilog2_exact(st.m);
        st.inv_m = 1.0f / (float)st.m;
        st.inv_nb = 1.0f / (float)st.nb;
        // padded-slot offsets: linear in the butterfly base when the same
        // off[r] works for every (q, j) of the stage (checked exhaustively)
        auto pad = [](int i) { return i + (i >> 4); };
        st.lin = R <= 16 ? 1 : 0;
        for (int r = 0; r < R && r < 16; ++r) st.off[r] = pad(r * st.m);
        for (int q = 0; q < L / Ls && st.lin; ++q)
            for (int j = 0; j < st.m && st.lin; ++j) {
                const int base = q * Ls + j;
                for (int r = 0; r < R; ++r)
                    if (pad(base + r * st.m) - pad(base) != st.off[r]) { st.lin = 0; break; }
            }
        Ls = st.m;
    }
    fp->Rlast = rad.back();
    fp->logRlast = ilog2_exact(fp->Rlast);
    return fp->logRlast >= 0;
}

template <typename T>
ls_status upload(ls_plan_s *p, void **dst, const void *src, size_t bytes)
{
    ls_status s = plan_alloc(p, dst, bytes);
    if (s != LS_OK) return s;
    // on the plan's stream, ahead of the kernels that read the table: a copy on
    // the legacy stream is not ordered with non-blocking streams, and a
    // pageable copy may return before its data has landed
    return cuda_status(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, p->stream));
}

template <typename T>
ls_status upload_tables(ls_plan_s *p)
{
    Geometry &g = p->g;
    std::vector<T> tA, tB, t4;
    if (!build_fft(g.N2, &g.fa, p->maxrA) || !build_fft(g.N1, &g.fb, p->maxrB))
        return LS_ERR_UNSUPPORTED;
    fill_root_table(tA, g.N2, 6);
    fill_root_table(tB, g.N1, 6);
    fill_root_table(t4, g.n, kTw4Bits);
    ls_status s;
    if ((s = upload<T>(p, &p->ws.twA, tA.data(), tA.size() * sizeof(T))) != LS_OK) return s;
    if ((s = upload<T>(p, &p->ws.twB, tB.data(), tB.size() * sizeof(T))) != LS_OK) return s;
    if ((s = upload<T>(p, &p->ws.tw4, t4.data(), t4.size() * sizeof(T))) != LS_OK) return s;

    // deconvolution table 1/phi_hat(k'), k' = 0 .. nf/2
    p->deconv_count = p->nf / 2 + 1;
    if ((s = plan_alloc(p, &p->ws.deconv, (size_t)p->deconv_count * sizeof(T))) != LS_OK) return s;
    std::vector<double> z, wpsi;
    es_quadrature(g.w, g.beta, z, wpsi);
    // The quadrature nodes stay with the plan (no free, which would
    // synchronise the device); the table kernels run on the plan's stream,
    // ahead of every launch that reads them (batch lanes wait for that stream).
    void *dq = nullptr;
    if ((s = plan_alloc(p, &dq, 2 * z.size() * sizeof(double))) != LS_OK) return s;
    double *dz = static_cast<double *>(dq), *dw = dz + z.size();
    cudaError_t e = cudaMemcpyAsync(dz, z.data(), z.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dw, wpsi.data(), wpsi.size() * sizeof(double), cudaMemcpyHostToDevice,
                            p->stream);
    if (e == cudaSuccess)
        e = launch_deconv_table<T>(g, p->ws.deconv, p->deconv_count, dz, dw, (int)z.size(),
                                   p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    // the same table in pass-B order (coalesced reads in pass B)
    if ((s = plan_alloc(p, &p->ws.deconv_slot, (size_t)g.n * sizeof(T))) != LS_OK) return s;
    return cuda_status(
        launch_deconv_slot<T>(g, p->ws.deconv_slot, p->ws.deconv, p->deconv_count, p->stream));
}

template <typename T>
ls_status plan_workspace(ls_plan_s *p, bool tables_only)
{
    if (tables_only) return upload_tables<T>(p);
    const Geometry &g = p->g;
    const size_t cx = sizeof(typename Cx<T>::type);
    ls_status s;
    if ((s = plan_alloc(p, &p->ws.H, 3 * (size_t)g.n * cx)) != LS_OK) return s;
    const size_t rec = point_record_bytes<T>() * (size_t)p->max_nd + 5 * 256;   // carve() alignment
    for (int i = 0; i < 2; ++i) {
        if ((s = plan_alloc(p, &p->ws.pts_raw[i], rec)) != LS_OK) return s;
        if ((s = plan_alloc(p, &p->ws.pts_sorted[i], rec)) != LS_OK) return s;
    }
    void *v;
    if ((s = plan_alloc(p, &v, sizeof(int) * 2 * (size_t)g.nbins)) != LS_OK) return s;
    p->ws.hist = static_cast<int *>(v);
    if ((s = plan_alloc(p, &v, sizeof(int) * 2 * ((size_t)g.nbins + 1))) != LS_OK) return s;
    p->ws.binstart = static_cast<int *>(v);
    if ((s = plan_alloc(p, &v, sizeof(int) * (size_t)chunk_hist_entries(p->max_nd, 1, g.nbins))) !=
        LS_OK)
        return s;
    p->ws.chist = static_cast<int *>(v);
    if ((s = plan_alloc(p, &v, sizeof(double) * 3 * (size_t)red_rows(p->max_nd, 1))) != LS_OK)
        return s;
    p->ws.partials = static_cast<double *>(v);
    if ((s = plan_alloc(p, &v, sizeof(double) * (size_t)p->max_nd)) != LS_OK) return s;
    p->ws.wts = static_cast<double *>(v);
    if ((s = plan_alloc(p, &v, 256)) != LS_OK) return s;
    p->ws.counter = static_cast<unsigned int *>(v);
    p->ws.status = reinterpret_cast<int *>(static_cast<char *>(v) + 64);
    if ((s = plan_alloc(p, &v, sizeof(Stats))) != LS_OK) return s;
    p->ws.stats = static_cast<Stats *>(v);
    cudaError_t e = cudaMemsetAsync(p->ws.counter, 0, 256, p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return upload_tables<T>(p);
}

bool is_device_pointer(const void *ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ls_status ensure_staging(ls_plan_s *p, double **buf, size_t count)
{
    if (*buf) return LS_OK;
    void *v;
    ls_status s = plan_alloc(p, &v, count * sizeof(double));
    if (s == LS_OK) *buf = static_cast<double *>(v);
    return s;
}

// Descriptor of one series: inputs at pt_off, records at rec_off, outputs at
// out_off, frequencies f0 + k df (k < nf), centre mode nf / 2.
SeriesDesc make_series(int64_t pt_off, int64_t rec_off, int64_t nd, int64_t out_off, int64_t nf,
                       double f0, double df)
{
    SeriesDesc d;
    d.pt_off = pt_off;
    d.y_off = pt_off;
    d.rec_off = rec_off;
    d.nd = nd;
    d.out_off = out_off;
    d.nf = nf;
    int neg;
    decompose_double(df, d.ph.df_m, d.ph.df_e, neg);
    decompose_double(f0, d.ph.f0_m, d.ph.f0_e, d.ph.f0_neg);
    d.ph.K0 = nf / 2;
    return d;
}

// Accumulate the oldest pending event set (waits for it).
cudaError_t drain_one_timing(ls_plan_s *p)
{
    const int idx = (p->t_head - p->t_pending + kTimingRing) % kTimingRing;
    cudaEvent_t *ev = p->tev.data() + (size_t)idx * kEvPerSet;
    cudaError_t e = cudaEventSynchronize(ev[kEvPerSet - 1]);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < LS_NUM_STAGES; ++s) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
        if (e != cudaSuccess) return e;
        p->t_acc[s] += ms;
    }
    p->t_count += 1;
    p->t_pending -= 1;
    return cudaSuccess;
}

void destroy_timing(ls_plan_s *p)
{
    for (cudaEvent_t e : p->tev) cudaEventDestroy(e);
    p->tev.clear();
    p->timing = false;
    p->t_pending = 0;
}

static_assert(LS_NO_FIT_MEAN == kModeNoFit && LS_NO_CENTER == kModeNoCenter,
              "model flags of the C-ABI and the kernels agree");

// The norm word: a normalisation in bits 0-7 plus model flags.
bool mode_supported(int norm)
{
    return (norm & ~(kModeNormMask | kModeNoFit | kModeNoCenter)) == 0 &&
           (norm & kModeNormMask) <= LS_NORM_PSD;
}

ls_status execute_impl(ls_plan_s *p, const double *t, const double *y, const double *dy,
                       int64_t nd, double f0, double df, int64_t nf, double eps, int norm,
                       double *power, double *sums)
{
    if (!p) return LS_ERR_ARG;
    if (!t || !y || (!power && !sums)) return LS_ERR_ARG;
    if (nd < 2 || nd > p->max_nd) return LS_ERR_ARG;
    if (nf < 1 || nf > p->nf) return LS_ERR_ARG;
    if (!(df > 0.0) || !isfinite(df) || !isfinite(f0)) return LS_ERR_ARG;
    if (!(eps >= p->eps * (1.0 - 1e-12)) || !isfinite(eps)) return LS_ERR_ARG;
    if (!mode_supported(norm)) return LS_ERR_UNSUPPORTED;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    cudaStream_t st = p->stream;
    cudaError_t e;
    ls_status s;

    const double *in[3] = {t, y, dy};
    const double *dev_in[3] = {t, y, dy};
    for (int i = 0; i < 3; ++i) {
        if (!in[i] || is_device_pointer(in[i])) continue;
        if ((s = ensure_staging(p, &p->stage_in, 3 * (size_t)p->max_nd)) != LS_OK) return s;
        double *dst = p->stage_in + (size_t)i * p->max_nd;
        e = cudaMemcpyAsync(dst, in[i], sizeof(double) * (size_t)nd, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_status(e);
        dev_in[i] = dst;
    }
    const bool host_power = power && !is_device_pointer(power);
    const bool host_sums = sums && !is_device_pointer(sums);
    double *dpow = power, *dsums = sums;
    if (host_power) {
        if ((s = ensure_staging(p, &p->stage_out, (size_t)p->nf)) != LS_OK) return s;
        dpow = p->stage_out;
    }
    if (host_sums) {
        if ((s = ensure_staging(p, &p->stage_sums, 6 * (size_t)p->nf)) != LS_OK) return s;
        dsums = p->stage_sums;
    }

    Batch bt;
    bt.S = 1;
    bt.many = nullptr;
    bt.one = make_series(0, 0, nd, 0, nf, f0, df);
    int nred = (int)((nd + 255) / 256);
    if (nred > p->nred) nred = p->nred;
    cudaEvent_t *ev = nullptr;
    if (p->timing) {
        if (p->t_pending == kTimingRing) {
            e = drain_one_timing(p);
            if (e != cudaSuccess) return cuda_status(e);
        }
        ev = p->tev.data() + (size_t)p->t_head * kEvPerSet;
        p->t_head = (p->t_head + 1) % kTimingRing;
        p->t_pending += 1;
    }
    e = (p->prec == LS_FP32)
            ? launch_pipeline<float>(p->g, p->ws, p->max_nd, bt, nd, dev_in[0], dev_in[1],
                                     dev_in[2], dpow, dsums, nred, st, ev, norm)
            : launch_pipeline<double>(p->g, p->ws, p->max_nd, bt, nd, dev_in[0], dev_in[1],
                                      dev_in[2], dpow, dsums, nred, st, ev, norm);
    if (e != cudaSuccess) return cuda_status(e);
    if (host_power || host_sums) {
        if (host_power) {
            e = cudaMemcpyAsync(power, dpow, sizeof(double) * (size_t)nf, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_status(e);
        }
        if (host_sums) {
            e = cudaMemcpyAsync(sums, dsums, 6 * sizeof(double) * (size_t)nf,
                                cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_status(e);
        }
        return ls_sync(p);
    }
    return LS_OK;
}

// ---------------------------------------------------------------------------
// ls_execute_batch support
// ---------------------------------------------------------------------------
void batch_free(ls_plan_s *p);

// Give lane workspace b its per-series arrays (once) and an arena of at least
// arena_need bytes (exact: no headroom).  st is the stream that last used b
// (synchronised before the arena is replaced); device errors of its launches go
// to the status word `status`.
ls_status reserve_ws(BatchWorkspace &b, cudaStream_t st, int nsm, int64_t arena_need,
                     bool exact = false)
{
    auto alloc = [&](void **ptr, size_t bytes) -> ls_status {
        cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            *ptr = nullptr;
            return cuda_status(e);
        }
        b.bytes += (int64_t)bytes;
        return LS_OK;
    };
    ls_status s;
    if (!b.stats) {
        void *v;
        if ((s = alloc(&v, sizeof(unsigned int) * 2 * kMaxBatchS)) != LS_OK) return s;
        b.allocs.push_back(v);
        b.counter = static_cast<unsigned int *>(v);
        // cleared on the stream that will run the lane's launches (a clear on the
        // legacy stream would not be ordered with the non-blocking lane streams)
        if (cudaMemsetAsync(b.counter, 0, sizeof(unsigned int) * 2 * kMaxBatchS, st) !=
            cudaSuccess)
            return LS_ERR_CUDA;
        if ((s = alloc(&v, sizeof(Stats) * kMaxBatchS)) != LS_OK) return s;
        b.allocs.push_back(v);
        b.stats = static_cast<Stats *>(v);
        if ((s = alloc(&v, sizeof(SeriesDesc) * kMaxBatchS)) != LS_OK) return s;
        b.allocs.push_back(v);
        b.desc = static_cast<SeriesDesc *>(v);
    }
    if (arena_need <= b.arena_bytes) return LS_OK;
    if (b.arena) {
        if (st) cudaStreamSynchronize(st);
        cudaFree(b.arena);
        b.bytes -= b.arena_bytes;
        b.arena = nullptr;
        b.arena_bytes = 0;
    }
    const int64_t want = exact ? arena_need : arena_need + arena_need / 4;
    if ((s = alloc(&b.arena, (size_t)want)) != LS_OK) return s;
    b.arena_bytes = want;
    return LS_OK;
}

void release_ws(BatchWorkspace &b)
{
    if (b.arena) cudaFree(b.arena);
    for (void *a : b.allocs) cudaFree(a);
    b = BatchWorkspace();
}

// The workspace of one launch: its buffers carved from the lane arena, the
// lane's per-series arrays, the plan's status word.
Workspace lane_workspace(const BatchWorkspace &b, const LaunchCarve &c, int *status)
{
    Workspace ws = {};
    char *a = static_cast<char *>(b.arena);
    ws.H = a + c.H;
    ws.pts_raw[0] = a + c.pts[0];
    ws.pts_raw[1] = a + c.pts[1];
    ws.pts_sorted[0] = a + c.pts[2];
    ws.pts_sorted[1] = a + c.pts[3];
    ws.hist = reinterpret_cast<int *>(a + c.hist);
    ws.binstart = reinterpret_cast<int *>(a + c.binstart);
    ws.chist = reinterpret_cast<int *>(a + c.chist);
    ws.wts = reinterpret_cast<double *>(a + c.wts);
    if (c.perm) {
        ws.perm = reinterpret_cast<int *>(a + c.perm);
        ws.cvals = a + c.cvals;
    }
    ws.partials = reinterpret_cast<double *>(a + c.partials);
    ws.counter = b.counter;
    ws.stats = b.stats;
    ws.status = status;
    return ws;
}

// Tile width (columns per pass-A block, also the bin width) and the largest
// FFT radix of pass A (length n2) and pass B (length n1), for both the planned
// path and the allocation-free one.  cols_req / maxr_req: requested values
// (0: automatic).  FFT schedules, automatic, from measurements on GB300: the
// double-float transforms of the FP64 path run faster with radix-8
// butterflies (fewer live registers) even where that adds a stage (pass A
// 5.2 -> 4.9 ms on a 1.9e7-cell grid, pass B 1.55x faster on 3.7e5 cells);
// on the FP32 path pass A keeps radix 16, and pass B takes radix 8 where
// that adds no stage (N1 = 512: 8, 8, 8 instead of 2, 16, 16; 8% faster).
void choose_tiling(int prec, int n1, int n2, int cols_req, int maxr_req, int *ba_out,
                   int *maxrA, int *maxrB)
{
    const size_t cx = prec == LS_FP32 ? 8 : 16;
    auto nstages = [](int L, int r) {
        std::vector<int> rad;
        return radix_schedule(L, rad, r) ? (int)rad.size() : 1 << 20;
    };
    if (maxr_req == 8 || maxr_req == 16) {
        *maxrA = *maxrB = maxr_req;
    } else if (prec == LS_FP64) {
        *maxrA = *maxrB = 8;
    } else {
        *maxrA = 16;
        *maxrB = nstages(n1, 8) <= nstages(n1, 16) ? 8 : 16;
    }
    // Tile width: the widest candidate whose two blocks fit an SM.  FP64 takes
    // at most 2 columns (measured: 2 columns ran pass A 1.8x faster than 8 on
    // a 3.7e5-cell grid, and the ragged FP64 batch 13% faster than the widest).
    static const int kColsF32[3] = {8, 4, 2}, kColsF64[1] = {2};
    const int *cands = prec == LS_FP64 ? kColsF64 : kColsF32;
    const int ncand = prec == LS_FP64 ? 1 : 3;
    int BA = 1;
    for (int i = 0; i < ncand; ++i) {
        const int cand = cands[i];
        if (n1 % cand == 0 && (size_t)cand * n2 * cx <= kSmemPairBudget && n1 / cand >= 2) {
            BA = cand;
            break;
        }
    }
    // Shared memory of a pass-A block of ba columns without cluster tables
    // (padded columns, root tables, slot table) plus 1 KB of margin.
    auto tile_bytes = [&](int ba) {
        std::vector<int> rad;
        if (!radix_schedule(n2, rad, *maxrA)) return (size_t)-1;
        const size_t nhi = (size_t)(n2 + 63) / 64;
        const size_t padded = (size_t)n2 + n2 / 16 + 1;
        return cx * ((size_t)ba * padded + (size_t)ba * (kAloStride + ahi_stride((int)nhi)) + 64 + nhi) +
               sizeof(int) * (size_t)(n2 / rad.back()) + (size_t)n2 + 1024;
    };
    // radix-8 stages need a larger slot table: keep 16 where it would not fit
    if (*maxrA == 8 && tile_bytes(BA) > kSmemOptinBytes) *maxrA = 16;
    // A requested tile width is taken where the grid can use it: at least two
    // bins, and the block within the opt-in shared memory (one block per SM
    // at the widest).
    if (cols_req > 0 && n1 % cols_req == 0 && n1 / cols_req >= 2 &&
        tile_bytes(cols_req) <= kSmemOptinBytes)
        BA = cols_req;
    *ba_out = BA;
}

// Plan (geometry, tables and, unless tables_only, the single-series workspace)
// for the parameters pp.
ls_status create_plan(ls_plan_t *out, int64_t max_nd, int64_t nf, double eps, int prec,
                      int device, void *stream, const PlanParams &pp, bool tables_only)
{
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? LS_ERR_ARG : LS_ERR_CUDA;
    }
    DeviceGuard guard(device);
    if (!guard.ok) return LS_ERR_CUDA;

    ls_plan_s *p = new (std::nothrow) ls_plan_s();
    if (!p) return LS_ERR_NOMEM;
    p->device = device;
    p->stream = static_cast<cudaStream_t>(stream);
    p->prec = prec;
    p->max_nd = max_nd;
    p->nf = nf;
    p->eps = eps;
    p->sigma = pp.sigma;
    p->upsampling = pp.upsampling;
    p->cols_req = pp.cols;
    p->maxr_req = pp.maxr;
    p->bytes = 0;
    p->stage_in = p->stage_out = p->stage_sums = nullptr;
    p->timing = false;
    p->t_head = p->t_pending = 0;
    for (double &a : p->t_acc) a = 0.0;
    p->t_count = 0;
    Geometry &g = p->g;
    g.n = pp.n;
    g.N1 = pp.n1;
    g.N2 = pp.n2;
    g.w = pp.w;
    g.beta = pp.beta;
    g.eps = eps;
    int BA = 1;
    choose_tiling(prec, pp.n1, pp.n2, pp.cols, pp.maxr, &BA, &p->maxrA, &p->maxrB);
    g.BA = BA;
    g.logBA = ilog2_exact(BA);
    g.nbins = pp.n1 / BA;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (nsm <= 0) nsm = 152;
    p->nsm = nsm;
    p->nred = 8 * nsm;
    ls_status s = (prec == LS_FP32) ? plan_workspace<float>(p, tables_only)
                                    : plan_workspace<double>(p, tables_only);
    // A plan the caller holds may later run on another stream (ls_set_stream):
    // its tables are complete when it is returned.  Batch classes (tables
    // only) are used on lanes that wait for the creating stream instead.
    if (s == LS_OK && !tables_only) s = cuda_status(cudaStreamSynchronize(p->stream));
    if (s != LS_OK) {
        if (p->stream) cudaStreamSynchronize(p->stream);
        plan_free(p);
        delete p;
        return s;
    }
    *out = p;
    return LS_OK;
}

void batch_free(ls_plan_s *p)
{
    for (int l = 0; l < kBatchLanes; ++l)
        if (p->lane_stream[l]) cudaStreamSynchronize(p->lane_stream[l]);
    for (BatchClass &c : p->classes) {
        plan_free(c.sub);
        delete c.sub;
    }
    p->classes.clear();
    for (int l = 0; l < kBatchLanes; ++l) {
        release_ws(p->bws[l]);
        if (p->lane_stream[l]) cudaStreamDestroy(p->lane_stream[l]);
        if (p->lane_done[l]) cudaEventDestroy(p->lane_done[l]);
        p->lane_stream[l] = nullptr;
        p->lane_done[l] = nullptr;
    }
    if (p->lane_start) cudaEventDestroy(p->lane_start);
    p->lane_start = nullptr;
}

// Start a batch call: the lanes wait for the work already queued on the
// plan's stream (their streams and events are created on first use).
ls_status lanes_begin(ls_plan_s *p)
{
    cudaError_t e;
    for (int l = 0; l < kBatchLanes; ++l) {
        if (!p->lane_stream[l]) {
            if ((e = cudaStreamCreateWithFlags(&p->lane_stream[l], cudaStreamNonBlocking)))
                return cuda_status(e);
            if ((e = cudaEventCreateWithFlags(&p->lane_done[l], cudaEventDisableTiming)))
                return cuda_status(e);
        }
    }
    if (!p->lane_start && (e = cudaEventCreateWithFlags(&p->lane_start, cudaEventDisableTiming)))
        return cuda_status(e);
    if ((e = cudaEventRecord(p->lane_start, p->stream))) return cuda_status(e);
    for (int l = 0; l < kBatchLanes; ++l)
        if ((e = cudaStreamWaitEvent(p->lane_stream[l], p->lane_start, 0))) return cuda_status(e);
    return LS_OK;
}

// End a batch call (also on error paths): the plan's stream waits for every lane.
struct LanesJoin {
    ls_plan_s *p;
    ~LanesJoin()
    {
        for (int l = 0; l < kBatchLanes; ++l) {
            if (!p->lane_stream[l]) continue;
            cudaEventRecord(p->lane_done[l], p->lane_stream[l]);
            cudaStreamWaitEvent(p->stream, p->lane_done[l], 0);
        }
    }
};

// Wait until no lane is using the class tables (before a class is rebuilt).
void lanes_sync(ls_plan_s *p)
{
    for (int l = 0; l < kBatchLanes; ++l)
        if (p->lane_stream[l]) cudaStreamSynchronize(p->lane_stream[l]);
}

// Tables-only sub-plan for the grid class of pp covering nf frequencies.
ls_status batch_class(ls_plan_s *p, const PlanParams &pp, int64_t nf, ls_plan_s **sub)
{
    for (BatchClass &c : p->classes) {
        if (c.pp.n == pp.n && c.pp.n1 == pp.n1 && c.pp.w == pp.w && c.pp.beta == pp.beta) {
            if (c.sub->nf >= nf) {
                *sub = c.sub;
                return LS_OK;
            }
            // the deconvolution table must reach nf/2: rebuild with the larger nf
            cudaStreamSynchronize(p->stream);
            lanes_sync(p);
            plan_free(c.sub);
            delete c.sub;
            ls_plan_t np;
            ls_status s = create_plan(&np, 2, nf, p->eps, p->prec, p->device, p->stream, pp, true);
            if (s != LS_OK) return s;
            c.sub = np;
            *sub = np;
            return LS_OK;
        }
    }
    ls_plan_t np;
    ls_status s = create_plan(&np, 2, nf, p->eps, p->prec, p->device, p->stream, pp, true);
    if (s != LS_OK) return s;
    p->classes.push_back(BatchClass{pp, np});
    *sub = np;
    return LS_OK;
}

// Reduction blocks per series of a batch launch: one per 256 points, at most
// about eight blocks per SM over the launch.
int batch_nred(const ls_plan_s *p, int S, int64_t max_nd)
{
    int nred = (int)((max_nd + 255) / 256);
    const int cap_red = (8 * p->nsm + S - 1) / S;
    if (nred > cap_red) nred = cap_red;
    return nred < 1 ? 1 : nred;
}

// Arena carve of a launch of S series over `points` records on a grid of n
// cells and nbins bins.
// A shared-times launch of S series of nd points each: H for the two common
// grids and one chunk of series grids, the common record sets and one
// series' bin tables, the sort permutation and weights (nd each), and the
// series' scalars c_i (S x nd).
LaunchCarve carve_shared(int prec, int64_t n, int nbins, int64_t S, int64_t nd)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t cx = prec == LS_FP32 ? 8 : 16;
    const size_t recb = prec == LS_FP32 ? point_record_bytes<float>() : point_record_bytes<double>();
    const size_t tb = prec == LS_FP32 ? sizeof(float) : sizeof(double);
    LaunchCarve c;
    size_t off = 0;
    c.H = off;
    off = al(off + cx * (size_t)n * (size_t)(2 + shared_chunk_series(n, cx, S)));
    const size_t rec = recb * (size_t)nd + 5 * 256;
    for (int i = 0; i < 4; ++i) {
        c.pts[i] = off;
        off = al(off + rec);
    }
    c.hist = off;
    off = al(off + sizeof(int) * 2 * (size_t)nbins);
    c.binstart = off;
    off = al(off + sizeof(int) * 2 * ((size_t)nbins + 1));
    c.chist = off;
    off = al(off + sizeof(int) * (size_t)chunk_hist_entries(nd, 1, nbins));
    c.perm = off;
    off = al(off + sizeof(int) * (size_t)nd);
    c.wts = off;
    off = al(off + sizeof(double) * (size_t)nd);
    c.cvals = off;
    off = al(off + tb * (size_t)S * (size_t)nd);
    c.partials = off;
    off = al(off + sizeof(double) * 3 * (size_t)red_rows(S * nd, S));
    c.bytes = off;
    return c;
}

LaunchCarve carve_for(int prec, int64_t n, int nbins, int64_t S, int64_t points, int shared)
{
    if (shared) return carve_shared(prec, n, nbins, S, points / (S > 0 ? S : 1));
    const size_t cx = prec == LS_FP32 ? 8 : 16;
    const size_t recb = prec == LS_FP32 ? point_record_bytes<float>() : point_record_bytes<double>();
    return carve_launch(n, nbins, cx, recb, S, points, 3 * S);
}

LaunchCarve launch_carve(const ls_plan_s *sub, int64_t S, int64_t points, int shared)
{
    return carve_for(sub->prec, sub->g.n, sub->g.nbins, S, points, shared);
}

// Series per launch of a shared-times batch: as many of the `left` series as
// fit lane_budget (at least one).
int64_t shared_launch_size(int prec, int64_t n, int nbins, int64_t nd, int64_t left,
                           int64_t lane_budget)
{
    int64_t S = 1;
    // (the common entry of the Stats and tickets takes slot S)
    while (S < kMaxBatchS - 1 && S < left &&
           (int64_t)carve_for(prec, n, nbins, S + 1, (S + 1) * nd, 1).bytes <= lane_budget)
        ++S;
    return S;
}

// Enqueue the pipeline of one batch launch on stream st: its buffers carved
// from lane workspace b (which holds them), tables of the class plan `sub`,
// descriptors already on the device.  Kernels and memsets only, so the launch
// can be recorded by stream capture.
template <typename T>
ls_status enqueue_batch(const BatchWorkspace &b, int *status, cudaStream_t st, const ls_plan_s *sub,
                        const Batch &bt, int64_t points, int64_t max_nd, int nred,
                        const double *t, const double *y, const double *dy, double *power,
                        int shared, int mode)
{
    const LaunchCarve c = launch_carve(sub, bt.S, points, shared);
    if ((int64_t)c.bytes > b.arena_bytes) return LS_ERR_ARG;
    Workspace ws = lane_workspace(b, c, status);
    ws.twA = sub->ws.twA;
    ws.twB = sub->ws.twB;
    ws.tw4 = sub->ws.tw4;
    ws.deconv = sub->ws.deconv;
    ws.deconv_slot = sub->ws.deconv_slot;
    if (shared)
        return cuda_status(launch_shared_pipeline<T>(sub->g, ws, bt, max_nd, t, y, dy, power,
                                                     nred, st, mode));
    return cuda_status(launch_pipeline<T>(sub->g, ws, points, bt, max_nd, t, y, dy, power,
                                          nullptr, nred, st, nullptr, mode));
}

template <typename T>
ls_status batch_launch(ls_plan_s *p, int lane, const ls_plan_s *sub, const std::vector<SeriesDesc> &descs,
                       int64_t points, int64_t max_nd, const double *t, const double *y,
                       const double *dy, double *power, int shared, int mode)
{
    const int S = (int)descs.size();
    const int nred = batch_nred(p, S, max_nd);
    const LaunchCarve c = launch_carve(sub, S, points, shared);
    ls_status s = reserve_ws(p->bws[lane], p->lane_stream[lane], p->nsm, (int64_t)c.bytes);
    if (s != LS_OK) return s;
    BatchWorkspace &b = p->bws[lane];
    cudaStream_t st = p->lane_stream[lane];
    cudaError_t e = cudaMemcpyAsync(b.desc, descs.data(), sizeof(SeriesDesc) * descs.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    Batch bt;
    bt.S = S;
    bt.many = b.desc;
    bt.one = descs[0];
    return enqueue_batch<T>(b, p->ws.status, st, sub, bt, points, max_nd, nred, t, y, dy, power,
                            shared, mode);
}

// Default batch budget: half of the free device memory, at most 8 GiB.
void init_batch_budget(ls_plan_s *p)
{
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    p->batch_budget = (int64_t)std::min<size_t>(fr / 2, (size_t)8 << 30);
}

// A grid class of a ragged batch call and the largest N_f among its series.
struct ClassSpec {
    PlanParams pp;
    int64_t nf_max;
};

// One launch of a ragged batch: series of one class (index cls) whose fine
// grids and point records fit the lane budget.
struct LaunchSpec {
    size_t cls;
    std::vector<SeriesDesc> descs;
    int64_t points = 0, max_nd = 0;
};

// Validate every series of a ragged batch, find its grid class (n, N1, w,
// beta of ls_choose_params), group the series by class (stable: series keep
// their order inside a class) and cut each class into launches of at most
// lane_budget bytes of grids and records.
ls_status split_batch(const ls_plan_s *p, int64_t nseries, const int64_t *offsets,
                      const double *f0, const double *df, const int64_t *nf,
                      const int64_t *out_offsets, double eps, int64_t lane_budget,
                      std::vector<ClassSpec> &classes, std::vector<LaunchSpec> &launches)
{
    struct Item {
        int64_t s;
        PlanParams pp;
    };
    std::vector<Item> items;
    items.reserve((size_t)nseries);
    for (int64_t s = 0; s < nseries; ++s) {
        const int64_t nd = offsets[s + 1] - offsets[s];
        if (offsets[s] < 0 || nd < 2 || nf[s] < 1 || out_offsets[s] < 0) return LS_ERR_ARG;
        if (!(df[s] > 0.0) || !isfinite(df[s]) || !isfinite(f0[s])) return LS_ERR_ARG;
        Item it;
        it.s = s;
        it.pp.upsampling = p->upsampling;
        it.pp.cols = p->cols_req;
        it.pp.maxr = p->maxr_req;
        ls_status st = ls_choose_params(nf[s], eps, p->prec, nd, p->upsampling, &it.pp.w,
                                        &it.pp.beta, &it.pp.n, &it.pp.n1, &it.pp.n2, &it.pp.sigma);
        if (st != LS_OK) return st;
        items.push_back(it);
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) {
        if (a.pp.n != b.pp.n) return a.pp.n > b.pp.n;
        if (a.pp.n1 != b.pp.n1) return a.pp.n1 < b.pp.n1;
        return a.pp.w < b.pp.w;
    });
    const size_t cx = p->prec == LS_FP32 ? 8 : 16;
    const size_t recb = p->prec == LS_FP32 ? point_record_bytes<float>() : point_record_bytes<double>();
    size_t i = 0;
    while (i < items.size()) {
        size_t j = i;
        int64_t nf_max = 0;
        while (j < items.size() && items[j].pp.n == items[i].pp.n && items[j].pp.n1 == items[i].pp.n1 &&
               items[j].pp.w == items[i].pp.w && items[j].pp.beta == items[i].pp.beta) {
            nf_max = std::max(nf_max, nf[items[j].s]);
            ++j;
        }
        classes.push_back(ClassSpec{items[i].pp, nf_max});
        int BA = 1, mA = 16, mB = 16;     // the class plan's tile width, hence its bins
        choose_tiling(p->prec, items[i].pp.n1, items[i].pp.n2, items[i].pp.cols, items[i].pp.maxr,
                      &BA, &mA, &mB);
        const int nbins = items[i].pp.n1 / BA;
        size_t k = i;
        while (k < j) {
            LaunchSpec L;
            L.cls = classes.size() - 1;
            while (k < j && (int)L.descs.size() < kMaxBatchS) {
                const int64_t s = items[k].s;
                const int64_t nd = offsets[s + 1] - offsets[s];
                const int64_t bytes = (int64_t)carve_launch(items[k].pp.n, nbins, cx, recb,
                                                            (int64_t)L.descs.size() + 1,
                                                            L.points + nd,
                                                            3 * ((int64_t)L.descs.size() + 1))
                                          .bytes;
                if (!L.descs.empty() && bytes > lane_budget) break;
                L.descs.push_back(make_series(offsets[s], L.points, nd, out_offsets[s], nf[s], f0[s],
                                              df[s]));
                L.points += nd;
                L.max_nd = std::max(L.max_nd, nd);
                ++k;
            }
            launches.push_back(std::move(L));
        }
        i = j;
    }
    return LS_OK;
}

// Build the prepared batch b from its classes and launches: class tables,
// per-lane workspaces sized for the launches each lane takes (round robin, as
// ls_execute_batch), and all descriptors in one device array.
template <typename T>
ls_status prepare_batch(ls_plan_s *p, ls_batch_s *b, const std::vector<ClassSpec> &classes,
                        const std::vector<LaunchSpec> &launches, int shared)
{
    for (const ClassSpec &c : classes) {
        ls_plan_t np = nullptr;
        ls_status s = create_plan(&np, 2, c.nf_max, p->eps, p->prec, p->device, p->stream, c.pp,
                                  true);
        if (s != LS_OK) return s;
        b->subs.push_back(np);
        b->bytes += np->bytes;
    }
    int64_t need[kBatchLanes] = {};   // arena bytes per lane (largest launch)
    bool used[kBatchLanes] = {};
    std::vector<SeriesDesc> all;
    int lane = 0;
    for (const LaunchSpec &L : launches) {
        const ls_plan_s *sub = b->subs[L.cls];
        PreparedLaunch pl;
        pl.lane = lane;
        pl.cls = L.cls;
        pl.S = (int)L.descs.size();
        pl.points = L.points;
        pl.max_nd = L.max_nd;
        pl.desc_off = all.size();
        pl.one = L.descs[0];
        pl.shared = shared;
        all.insert(all.end(), L.descs.begin(), L.descs.end());
        used[lane] = true;
        need[lane] = std::max(need[lane], (int64_t)launch_carve(sub, pl.S, pl.points, shared).bytes);
        b->launches.push_back(pl);
        lane = (lane + 1) % kBatchLanes;
    }
    for (int l = 0; l < kBatchLanes; ++l) {
        if (!used[l]) continue;
        ls_status s = reserve_ws(b->bws[l], p->stream, p->nsm, need[l], true);
        if (s != LS_OK) return s;
        b->bytes += b->bws[l].bytes;
    }
    void *v = nullptr;
    const size_t db = sizeof(SeriesDesc) * all.size();
    cudaError_t e = cudaMalloc(&v, db);
    if (e != cudaSuccess) return cuda_status(e);
    b->desc_all = static_cast<SeriesDesc *>(v);
    b->bytes += (int64_t)db;
    // the class tables, counter clears and descriptors were enqueued on the
    // plan's stream: complete before any run, whatever stream it comes on
    cudaError_t e2 = cudaMemcpyAsync(b->desc_all, all.data(), db, cudaMemcpyHostToDevice, p->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(p->stream);
    return cuda_status(e2);
}

void batch_release(ls_batch_s *b)
{
    for (ls_plan_s *sp : b->subs) {
        plan_free(sp);
        delete sp;
    }
    b->subs.clear();
    for (BatchWorkspace &w : b->bws) release_ws(w);
    if (b->desc_all) cudaFree(b->desc_all);
    b->desc_all = nullptr;
}

// Validation shared by the batch entry points (series-independent arguments).
ls_status check_batch_call(const ls_plan_s *p, double eps, int norm)
{
    if (!mode_supported(norm)) return LS_ERR_UNSUPPORTED;
    if (!(eps >= p->eps * (1.0 - 1e-12)) || !isfinite(eps)) return LS_ERR_ARG;
    return LS_OK;
}

ls_status finish_prepare(ls_plan_s *p, ls_batch_s *b, const std::vector<ClassSpec> &classes,
                         const std::vector<LaunchSpec> &launches, int shared, ls_batch_t *out)
{
    ls_status st = (p->prec == LS_FP32) ? prepare_batch<float>(p, b, classes, launches, shared)
                                        : prepare_batch<double>(p, b, classes, launches, shared);
    if (st == LS_OK) {
        // the lanes' streams and events exist before any run (none is created
        // while a run is being recorded)
        st = lanes_begin(p);
        LanesJoin join{p};
    }
    if (st != LS_OK) {
        batch_release(b);
        delete b;
        return st;
    }
    p->batches.push_back(b);
    *out = b;
    return LS_OK;
}

}  // namespace

namespace nls {
// Stage descriptors of a length-L FFT for callers outside this file.
bool fft_plan_for_length(int L, FftPlan *fp, int maxr) { return build_fft(L, fp, maxr); }

void plan_tiling(int prec, int n1, int n2, int *ba, int *maxrA, int *maxrB)
{
    choose_tiling(prec, n1, n2, 0, 0, ba, maxrA, maxrB);
}

int es_quadrature_into(int w, double beta, double *z, double *wpsi, int cap)
{
    return es_quadrature_fill(w, beta, z, wpsi, cap);
}
}  // namespace nls

extern "C" {

const char *ls_status_str(ls_status s)
{
    switch (s) {
    case LS_OK: return "ok";
    case LS_ERR_ARG: return "invalid argument or input values";
    case LS_ERR_NOMEM: return "out of memory";
    case LS_ERR_CUDA: return "CUDA runtime error";
    case LS_ERR_TIMEOUT: return "device-side wait timed out";
    case LS_ERR_DEGENERATE: return "degenerate input: the weighted variance of y is zero";
    case LS_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

ls_status ls_choose_params(int64_t nf, double eps, int prec, int64_t max_nd, double upsampling,
                           int32_t *width, double *beta, int64_t *n, int32_t *n1, int32_t *n2,
                           double *sigma_out)
{
    if (nf < 1 || !(eps >= 1e-14 && eps <= 1e-1)) return LS_ERR_ARG;
    if (prec != LS_FP32 && prec != LS_FP64) return LS_ERR_ARG;
    if (prec == LS_FP32 && eps < 1e-7) return LS_ERR_ARG;
    if (max_nd < 1) max_nd = 1;
    if (!(upsampling == 0.0 || upsampling == 2.0 || upsampling == 1.5)) return LS_ERR_ARG;
    // Candidates: sigma = 2 always; sigma = 1.5 for eps >= 1e-10.  Auto picks
    // the smaller modelled cost: fine-grid cells (FFT and HBM traffic) plus
    // half a cell per kernel evaluation of the spread.
    double best_cost = 1e300;
    ls_status st = LS_ERR_UNSUPPORTED;
    for (double sg : {2.0, 1.5}) {
        if (upsampling != 0.0 && sg != upsampling) continue;
        if (sg != 2.0 && eps < 1e-10) continue;
        int w;
        double b;
        if (!es_params(eps, sg, &w, &b)) continue;
        int64_t nn;
        int a1, a2;
        if (choose_grid(nf, sg, w, prec, &nn, &a1, &a2) != LS_OK) continue;
        const double cost = (double)nn + 0.5 * (double)max_nd * w;
        if (cost < best_cost) {
            best_cost = cost;
            st = LS_OK;
            if (width) *width = w;
            if (beta) *beta = b;
            if (n) *n = nn;
            if (n1) *n1 = a1;
            if (n2) *n2 = a2;
            if (sigma_out) *sigma_out = sg;
        }
    }
    return st;
}

double ls_kernel_ft(double k, int64_t n, int32_t width, double beta)
{
    std::vector<double> z, wpsi;
    es_quadrature(width, beta, z, wpsi);
    double s = 0.0;
    for (size_t i = 0; i < z.size(); ++i) s += wpsi[i] * cos(M_PI * k * width * z[i] / (double)n);
    return width * s;
}

ls_status ls_plan(ls_plan_t *out, int64_t max_nd, int64_t nf, double eps, int prec, int device,
                  void *stream)
{
    return ls_plan_ex(out, max_nd, nf, eps, prec, device, stream, nullptr);
}

ls_status ls_plan_ex(ls_plan_t *out, int64_t max_nd, int64_t nf, double eps, int prec, int device,
                     void *stream, const ls_plan_opts *opts)
{
    if (!out) return LS_ERR_ARG;
    *out = nullptr;
    if (max_nd < 2 || max_nd > ((int64_t)1 << 30)) return LS_ERR_ARG;
    PlanParams pp;
    pp.upsampling = opts ? opts->upsampling : 0.0;
    if (opts) {
        const int c = opts->cols_per_block, r = opts->fft_max_radix;
        if (!(c == 0 || c == 1 || c == 2 || c == 4 || c == 8)) return LS_ERR_ARG;
        if (!(r == 0 || r == 8 || r == 16)) return LS_ERR_ARG;
        pp.cols = c;
        pp.maxr = r;
    }
    ls_status s = ls_choose_params(nf, eps, prec, max_nd, pp.upsampling, &pp.w, &pp.beta, &pp.n,
                                   &pp.n1, &pp.n2, &pp.sigma);
    if (s != LS_OK) return s;
    s = create_plan(out, max_nd, nf, eps, prec, device, stream, pp, false);
    if (s == LS_OK && opts && opts->batch_workspace_bytes > 0)
        (*out)->batch_budget = (int64_t)opts->batch_workspace_bytes;
    return s;
}

ls_status ls_plan_reserve_batch(ls_plan_t p)
{
    if (!p) return LS_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    if (p->batch_budget <= 0) init_batch_budget(p);
    ls_status st = lanes_begin(p);
    if (st != LS_OK) return st;
    LanesJoin join{p};
    const int64_t lane_budget = p->batch_budget / kBatchLanes;
    for (int l = 0; l < kBatchLanes; ++l) {
        st = reserve_ws(p->bws[l], p->lane_stream[l], p->nsm, lane_budget, true);
        if (st != LS_OK) return st;
    }
    return LS_OK;
}

ls_status ls_execute_batch(ls_plan_t p, int64_t nseries, const int64_t *offsets, const double *t,
                           const double *y, const double *dy, const double *f0, const double *df,
                           const int64_t *nf, const int64_t *out_offsets, double eps, int norm,
                           double *power)
{
    if (!p || nseries < 0 || !offsets || !f0 || !df || !nf || !out_offsets) return LS_ERR_ARG;
    if (nseries == 0) return LS_OK;
    if (!t || !y || !power) return LS_ERR_ARG;
    if (!mode_supported(norm)) return LS_ERR_UNSUPPORTED;
    if (!(eps >= p->eps * (1.0 - 1e-12)) || !isfinite(eps)) return LS_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    if (!is_device_pointer(t) || !is_device_pointer(y) || !is_device_pointer(power) ||
        (dy && !is_device_pointer(dy)))
        return LS_ERR_ARG;
    if (p->batch_budget <= 0) init_batch_budget(p);
    std::vector<ClassSpec> classes;
    std::vector<LaunchSpec> launches;
    ls_status st = split_batch(p, nseries, offsets, f0, df, nf, out_offsets, eps,
                               p->batch_budget / kBatchLanes, classes, launches);
    if (st != LS_OK) return st;
    std::vector<ls_plan_s *> subs(classes.size(), nullptr);
    for (size_t c = 0; c < classes.size(); ++c)
        if ((st = batch_class(p, classes[c].pp, classes[c].nf_max, &subs[c])) != LS_OK) return st;
    if ((st = lanes_begin(p)) != LS_OK) return st;
    LanesJoin join{p};
    int lane = 0;
    for (const LaunchSpec &L : launches) {
        st = (p->prec == LS_FP32)
                 ? batch_launch<float>(p, lane, subs[L.cls], L.descs, L.points, L.max_nd, t, y, dy,
                                       power, 0, norm)
                 : batch_launch<double>(p, lane, subs[L.cls], L.descs, L.points, L.max_nd, t, y, dy,
                                        power, 0, norm);
        if (st != LS_OK) return st;
        lane = (lane + 1) % kBatchLanes;
    }
    return LS_OK;
}

ls_status ls_execute_batch_shared(ls_plan_t p, int64_t nseries, int64_t nd, const double *t,
                                  const double *Y, const double *dy, double f0, double df,
                                  int64_t nf, double eps, int norm, double *power)
{
    if (!p || nseries < 0) return LS_ERR_ARG;
    if (nseries == 0) return LS_OK;
    if (!t || !Y || !power || nd < 2 || nf < 1) return LS_ERR_ARG;
    if (!(df > 0.0) || !isfinite(df) || !isfinite(f0)) return LS_ERR_ARG;
    if (!mode_supported(norm)) return LS_ERR_UNSUPPORTED;
    if (!(eps >= p->eps * (1.0 - 1e-12)) || !isfinite(eps)) return LS_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    if (!is_device_pointer(t) || !is_device_pointer(Y) || !is_device_pointer(power) ||
        (dy && !is_device_pointer(dy)))
        return LS_ERR_ARG;
    PlanParams pp;
    pp.upsampling = p->upsampling;
    pp.cols = p->cols_req;
    pp.maxr = p->maxr_req;
    ls_status st = ls_choose_params(nf, eps, p->prec, nd, p->upsampling, &pp.w, &pp.beta, &pp.n,
                                    &pp.n1, &pp.n2, &pp.sigma);
    if (st != LS_OK) return st;
    ls_plan_s *sub = nullptr;
    if ((st = batch_class(p, pp, nf, &sub)) != LS_OK) return st;
    if (p->batch_budget <= 0) init_batch_budget(p);
    const int64_t lane_budget = p->batch_budget / kBatchLanes;
    ls_status lst = lanes_begin(p);
    if (lst != LS_OK) return lst;
    LanesJoin join{p};
    int lane = 0;
    int64_t s0 = 0;
    while (s0 < nseries) {
        // series per launch within the budget: H holds S + 2 grids
        const int64_t S = shared_launch_size(p->prec, sub->g.n, sub->g.nbins, nd, nseries - s0,
                                             lane_budget);
        std::vector<SeriesDesc> descs;
        descs.reserve((size_t)S);
        for (int64_t k = 0; k < S; ++k) {
            SeriesDesc d = make_series(0, k * nd, nd, (s0 + k) * nf, nf, f0, df);
            d.y_off = (s0 + k) * nd;
            descs.push_back(d);
        }
        st = (p->prec == LS_FP32)
                 ? batch_launch<float>(p, lane, sub, descs, S * nd, nd, t, Y, dy, power, 1, norm)
                 : batch_launch<double>(p, lane, sub, descs, S * nd, nd, t, Y, dy, power, 1, norm);
        if (st != LS_OK) return st;
        lane = (lane + 1) % kBatchLanes;
        s0 += S;
    }
    return LS_OK;
}

ls_status ls_batch_prepare(ls_plan_t p, ls_batch_t *out, int64_t nseries, const int64_t *offsets,
                           const double *f0, const double *df, const int64_t *nf,
                           const int64_t *out_offsets, double eps, int norm)
{
    if (!out) return LS_ERR_ARG;
    *out = nullptr;
    if (!p || nseries < 1 || !offsets || !f0 || !df || !nf || !out_offsets) return LS_ERR_ARG;
    ls_status st = check_batch_call(p, eps, norm);
    if (st != LS_OK) return st;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    if (p->batch_budget <= 0) init_batch_budget(p);
    std::vector<ClassSpec> classes;
    std::vector<LaunchSpec> launches;
    st = split_batch(p, nseries, offsets, f0, df, nf, out_offsets, eps,
                     p->batch_budget / kBatchLanes, classes, launches);
    if (st != LS_OK) return st;
    ls_batch_s *b = new (std::nothrow) ls_batch_s();
    if (!b) return LS_ERR_NOMEM;
    b->plan = p;
    b->norm = norm;
    return finish_prepare(p, b, classes, launches, 0, out);
}

ls_status ls_batch_prepare_shared(ls_plan_t p, ls_batch_t *out, int64_t nseries, int64_t nd,
                                  double f0, double df, int64_t nf, double eps, int norm)
{
    if (!out) return LS_ERR_ARG;
    *out = nullptr;
    if (!p || nseries < 1 || nd < 2 || nf < 1) return LS_ERR_ARG;
    if (!(df > 0.0) || !isfinite(df) || !isfinite(f0)) return LS_ERR_ARG;
    ls_status st = check_batch_call(p, eps, norm);
    if (st != LS_OK) return st;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    PlanParams pp;
    pp.upsampling = p->upsampling;
    pp.cols = p->cols_req;
    pp.maxr = p->maxr_req;
    st = ls_choose_params(nf, eps, p->prec, nd, p->upsampling, &pp.w, &pp.beta, &pp.n, &pp.n1,
                          &pp.n2, &pp.sigma);
    if (st != LS_OK) return st;
    if (p->batch_budget <= 0) init_batch_budget(p);
    const int64_t lane_budget = p->batch_budget / kBatchLanes;
    std::vector<ClassSpec> classes{ClassSpec{pp, nf}};
    std::vector<LaunchSpec> launches;
    int BA = 1, mA = 16, mB = 16;     // the class plan's tile width, hence its bins
    choose_tiling(p->prec, pp.n1, pp.n2, pp.cols, pp.maxr, &BA, &mA, &mB);
    for (int64_t s0 = 0; s0 < nseries;) {
        // series per launch within the lane budget (as ls_execute_batch_shared)
        const int64_t S = shared_launch_size(p->prec, pp.n, pp.n1 / BA, nd, nseries - s0,
                                             lane_budget);
        LaunchSpec L;
        L.cls = 0;
        L.points = S * nd;
        L.max_nd = nd;
        for (int64_t k = 0; k < S; ++k) {
            SeriesDesc d = make_series(0, k * nd, nd, (s0 + k) * nf, nf, f0, df);
            d.y_off = (s0 + k) * nd;
            L.descs.push_back(d);
        }
        launches.push_back(std::move(L));
        s0 += S;
    }
    ls_batch_s *b = new (std::nothrow) ls_batch_s();
    if (!b) return LS_ERR_NOMEM;
    b->plan = p;
    b->norm = norm;
    return finish_prepare(p, b, classes, launches, 1, out);
}

ls_status ls_batch_run(ls_batch_t b, const double *t, const double *y, const double *dy,
                       double *power)
{
    if (!b || !b->plan || !t || !y || !power) return LS_ERR_ARG;
    ls_plan_s *p = b->plan;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    if (!is_device_pointer(t) || !is_device_pointer(y) || !is_device_pointer(power) ||
        (dy && !is_device_pointer(dy)))
        return LS_ERR_ARG;
    ls_status st = lanes_begin(p);
    if (st != LS_OK) return st;
    LanesJoin join{p};
    for (const PreparedLaunch &L : b->launches) {
        Batch bt;
        bt.S = L.S;
        bt.many = b->desc_all + L.desc_off;
        bt.one = L.one;
        const int nred = batch_nred(p, L.S, L.max_nd);
        const ls_plan_s *sub = b->subs[L.cls];
        cudaStream_t ls = p->lane_stream[L.lane];
        st = (p->prec == LS_FP32)
                 ? enqueue_batch<float>(b->bws[L.lane], p->ws.status, ls, sub, bt, L.points,
                                        L.max_nd, nred, t, y, dy, power, L.shared, b->norm)
                 : enqueue_batch<double>(b->bws[L.lane], p->ws.status, ls, sub, bt, L.points,
                                         L.max_nd, nred, t, y, dy, power, L.shared, b->norm);
        if (st != LS_OK) return st;
    }
    return LS_OK;
}

ls_status ls_batch_describe(ls_batch_t b, int64_t *launches, int64_t *classes, int64_t *bytes)
{
    if (!b || !b->plan) return LS_ERR_ARG;
    if (launches) *launches = (int64_t)b->launches.size();
    if (classes) *classes = (int64_t)b->subs.size();
    if (bytes) *bytes = b->bytes;
    return LS_OK;
}

ls_status ls_batch_destroy(ls_batch_t b)
{
    if (!b) return LS_ERR_ARG;
    if (ls_plan_s *p = b->plan) {
        DeviceGuard guard(p->device);
        cudaStreamSynchronize(p->stream);
        lanes_sync(p);
        batch_release(b);
        p->batches.erase(std::remove(p->batches.begin(), p->batches.end(), b), p->batches.end());
    }
    delete b;
    return LS_OK;
}

ls_status ls_kernel_launches(int64_t *count)
{
    if (!count) return LS_ERR_ARG;
    *count = (int64_t)pipeline_kernel_count();
    return LS_OK;
}

ls_status ls_selftest_kernel_eval(double beta, int n, int device, double *max_abs_err)
{
    if (!max_abs_err || n < 2 || n > (1 << 24) || !(beta > 0.0) || !(beta < 100.0))
        return LS_ERR_ARG;
    DeviceGuard guard(device);
    if (!guard.ok) return LS_ERR_CUDA;
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(double) * (size_t)n);
    if (e != cudaSuccess) return LS_ERR_NOMEM;
    e = launch_kernel_eval_pair(n, beta, d, d + n, 0);
    std::vector<double> h(2 * (size_t)n);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.data(), d, 2 * sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_status(e);
    double worst = 0.0;
    for (int i = 0; i < n; ++i) {
        const double d = fabs(h[(size_t)i] - h[(size_t)n + i]);
        if (!(d <= worst)) worst = d;
    }
    *max_abs_err = worst;
    return LS_OK;
}

ls_status ls_selftest_double_assembly(int64_t n, uint64_t seed, int device, int64_t *mismatches)
{
    if (!mismatches || n < 1 || n > ((int64_t)1 << 32)) return LS_ERR_ARG;
    DeviceGuard guard(device);
    if (!guard.ok) return LS_ERR_CUDA;
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
    if (e != cudaSuccess) return LS_ERR_NOMEM;
    unsigned long long h = 0;
    e = cudaMemset(d, 0, sizeof h);
    if (e == cudaSuccess) e = launch_ff_assembly_check((long long)n, (unsigned long long)seed, d, 0);
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_status(e);
    *mismatches = (int64_t)h;
    return LS_OK;
}

ls_status ls_set_stream(ls_plan_t p, void *stream)
{
    if (!p) return LS_ERR_ARG;
    p->stream = static_cast<cudaStream_t>(stream);
    return LS_OK;
}

ls_status ls_execute(ls_plan_t p, const double *t, const double *y, const double *dy, int64_t nd,
                     double f0, double df, int64_t nf, double eps, int norm, double *power)
{
    if (!power) return LS_ERR_ARG;
    return execute_impl(p, t, y, dy, nd, f0, df, nf, eps, norm, power, nullptr);
}

ls_status ls_execute_sums(ls_plan_t p, const double *t, const double *y, const double *dy,
                          int64_t nd, double f0, double df, int64_t nf, double eps, int norm,
                          double *power, double *sums)
{
    if (!sums) return LS_ERR_ARG;
    return execute_impl(p, t, y, dy, nd, f0, df, nf, eps, norm, power, sums);
}

ls_status ls_sync(ls_plan_t p)
{
    if (!p) return LS_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    // Everything on the plan's own stream: a copy on the legacy default stream
    // would also wait for work that other plans have queued on other streams.
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, p->ws.status, sizeof(int), cudaMemcpyDeviceToHost,
                                    p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (h) {
        e = cudaMemsetAsync(p->ws.status, 0, sizeof(int), p->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (h & kStatBadInput) return LS_ERR_ARG;
    if (h & kStatDegenerate) return LS_ERR_DEGENERATE;
    return LS_OK;
}

ls_status ls_plan_describe(ls_plan_t p, ls_plan_info *info)
{
    if (!p || !info) return LS_ERR_ARG;
    info->nf = p->nf;
    info->max_nd = p->max_nd;
    info->n = p->g.n;
    info->n1 = p->g.N1;
    info->n2 = p->g.N2;
    info->width = p->g.w;
    info->prec = p->prec;
    info->beta = p->g.beta;
    info->eps = p->eps;
    info->sigma = p->sigma;
    info->workspace_bytes = p->bytes;
    int64_t bb = 0;
    for (int l = 0; l < kBatchLanes; ++l) bb += p->bws[l].bytes;
    for (const BatchClass &c : p->classes) bb += c.sub->bytes;
    info->batch_bytes = bb;
    info->cols_per_block = p->g.BA;
    int r = 0;
    for (const FftPlan *f : {&p->g.fa, &p->g.fb})
        for (int k = 0; k < f->nstages; ++k) {
            const int R = f->st[k].R;
            if ((R & (R - 1)) == 0 && R > r) r = R;
        }
    info->fft_max_radix = r;
    return LS_OK;
}

ls_status ls_timing_enable(ls_plan_t p, int enable)
{
    if (!p) return LS_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    if (!enable) {
        destroy_timing(p);
        return LS_OK;
    }
    if (p->timing) return LS_OK;
    p->tev.assign((size_t)kTimingRing * kEvPerSet, nullptr);
    for (auto &e : p->tev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            destroy_timing(p);
            return LS_ERR_CUDA;
        }
    }
    p->timing = true;
    p->t_head = p->t_pending = 0;
    for (double &a : p->t_acc) a = 0.0;
    p->t_count = 0;
    return LS_OK;
}

ls_status ls_timing_report(ls_plan_t p, double *ms, int64_t *count)
{
    if (!p || !ms) return LS_ERR_ARG;
    if (!p->timing) return LS_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return LS_ERR_CUDA;
    while (p->t_pending > 0) {
        cudaError_t e = drain_one_timing(p);
        if (e != cudaSuccess) return cuda_status(e);
    }
    for (int s = 0; s < LS_NUM_STAGES; ++s) {
        ms[s] = p->t_acc[s];
        p->t_acc[s] = 0.0;
    }
    if (count) *count = p->t_count;
    p->t_count = 0;
    return LS_OK;
}

ls_status ls_destroy(ls_plan_t p)
{
    if (!p) return LS_ERR_ARG;
    {
        DeviceGuard guard(p->device);
        cudaStreamSynchronize(p->stream);
        // batches still prepared on this plan lose their device memory and
        // become inert handles (ls_batch_run refuses them; ls_batch_destroy
        // only frees the handle)
        lanes_sync(p);
        for (ls_batch_s *b : p->batches) {
            batch_release(b);
            b->plan = nullptr;
        }
        p->batches.clear();
        destroy_timing(p);
        batch_free(p);
        plan_free(p);
    }
    delete p;
    return LS_OK;
}

}  // extern "C"
