// Periodogram entry point that allocates no memory: ls_execute_noalloc.
//
// Who needs it: callers that must not allocate device memory themselves or
// through a library -- processes whose device memory is owned by another
// allocator (a framework's caching allocator, or a fixed arena that a raw
// cudaMalloc would fragment or exceed), and loops that cannot afford the
// device-wide synchronisation a cudaMalloc or cudaFree may bring.  Such
// callers cannot create an ls_plan (ls_plan allocates its workspace), so this
// entry point runs the same pipeline on a fixed scratch area that the library
// reserves when it is loaded: a file-scope __device__ array, which every GPU
// that loads the library holds until the process exits.
//
// The call is synchronous: it copies the deconvolution quadrature from a host
// stack buffer, waits for its stream and reads the device-side status word
// back.  It therefore cannot run while its stream is being captured into a
// CUDA graph.
//
// Set-up: the host cannot use the array's name as a device address (in host
// code it names a host-side stand-in).  The first call on each device, with
// that device current, resolves the address with cudaGetSymbolAddress and
// keeps it for the life of the process.  A cudaDeviceReset tears down the
// context that address belongs to, so do not call this entry point on a
// device after resetting it.
//
// Sharing: every call uses the same array and leaves its contents behind.
// Counters and status words that must start at zero are cleared at the start
// of each call; calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the
// caller.
#include <math.h>
#include <mutex>

#include "ls_internal.cuh"

namespace nls {

// Fixed scratch: 8 MiB per device.
constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices];   // device address of g_noalloc_scratch, per device

// Resolve the scratch address for the current device (once per device).
cudaError_t scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

// Bump allocator over the scratch array (offsets only; nothing is allocated).
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return at;
    }
};

// exp(2 pi i p / L) for the two-level root table: entries p < 2^bits, then
// (L + 2^bits - 1) >> bits entries of p = i 2^bits.  FP64 sincospi, rounded to T.
template <typename T>
__global__ void k_root_table(T *out, int64_t L, int bits)
{
    const int64_t lo = (int64_t)1 << bits;
    const int64_t count = lo + ((L + lo - 1) >> bits);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = (i < lo) ? i : (i - lo) * lo;
        p %= L;
        double s, c;
        sincospi(2.0 * (double)p / (double)L, &s, &c);
        out[2 * i] = (T)c;
        out[2 * i + 1] = (T)s;
    }
}

constexpr int kMaxQuad = 64;   // nodes of the deconvolution quadrature

bool device_pointer(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
ls_status run_noalloc(unsigned char *base, const double *t, const double *y, const double *dy,
                      int64_t nd, double f0, double df, int64_t nf, double eps, double *power,
                      cudaStream_t st)
{
    using V = typename Cx<T>::type;
    const int prec = sizeof(T) == 4 ? LS_FP32 : LS_FP64;
    Geometry g;
    int32_t w, n1, n2;
    double beta, sigma;
    int64_t n;
    ls_status s = ls_choose_params(nf, eps, prec, nd, 0.0, &w, &beta, &n, &n1, &n2, &sigma);
    if (s != LS_OK) return s;
    g.n = n;
    g.N1 = n1;
    g.N2 = n2;
    g.w = w;
    g.beta = beta;
    g.eps = eps;
    // the same tile width and FFT schedules as a plan for this request
    int BA = 1, maxrA = 16, maxrB = 16;
    plan_tiling(prec, n1, n2, &BA, &maxrA, &maxrB);
    if (!fft_plan_for_length(n2, &g.fa, maxrA) || !fft_plan_for_length(n1, &g.fb, maxrB))
        return LS_ERR_UNSUPPORTED;
    g.BA = BA;
    g.logBA = BA == 8 ? 3 : BA == 4 ? 2 : BA == 2 ? 1 : 0;
    g.nbins = n1 / BA;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 152;
    int nred = (int)((nd + 255) / 256);
    if (nred > 8 * nsm) nred = 8 * nsm;

    // Layout inside the scratch array.
    Carver c;
    const size_t o_counter = c.take(256);
    const size_t o_stats = c.take(sizeof(Stats));
    const size_t o_partials = c.take(sizeof(double) * 3 * (size_t)red_rows(nd, 1));
    const size_t o_wts = c.take(sizeof(double) * (size_t)nd);
    const size_t o_hist = c.take(sizeof(int) * 2 * (size_t)g.nbins);
    const size_t o_binstart = c.take(sizeof(int) * 2 * ((size_t)g.nbins + 1));
    const size_t o_chist = c.take(sizeof(int) * (size_t)chunk_hist_entries(nd, 1, g.nbins));
    const size_t rec = point_record_bytes<T>() * (size_t)nd + 5 * 256;   // carve() alignment
    size_t o_pts[4];
    for (int i = 0; i < 4; ++i) o_pts[i] = c.take(rec);
    const size_t o_H = c.take(3 * (size_t)n * sizeof(V));
    const size_t o_twA = c.take(sizeof(V) * (64 + ((size_t)n2 + 63) / 64));
    const size_t o_twB = c.take(sizeof(V) * (64 + ((size_t)n1 + 63) / 64));
    const size_t o_tw4 = c.take(sizeof(V) * ((1u << kTw4Bits) + ((size_t)n >> kTw4Bits) + 1));
    const int64_t ndeconv = nf / 2 + 1;
    const size_t o_deconv = c.take(sizeof(T) * (size_t)ndeconv);
    const size_t o_deconv_slot = c.take(sizeof(T) * (size_t)n);
    const size_t o_quad = c.take(sizeof(double) * 2 * kMaxQuad);
    if (c.off > kNoallocScratchBytes) return LS_ERR_UNSUPPORTED;

    Workspace ws = {};
    ws.counter = reinterpret_cast<unsigned int *>(base + o_counter);
    ws.status = reinterpret_cast<int *>(base + o_counter + 64);
    ws.stats = reinterpret_cast<Stats *>(base + o_stats);
    ws.partials = reinterpret_cast<double *>(base + o_partials);
    ws.wts = reinterpret_cast<double *>(base + o_wts);
    ws.hist = reinterpret_cast<int *>(base + o_hist);
    ws.binstart = reinterpret_cast<int *>(base + o_binstart);
    ws.chist = reinterpret_cast<int *>(base + o_chist);
    ws.pts_raw[0] = base + o_pts[0];
    ws.pts_raw[1] = base + o_pts[1];
    ws.pts_sorted[0] = base + o_pts[2];
    ws.pts_sorted[1] = base + o_pts[3];
    ws.H = base + o_H;
    ws.twA = base + o_twA;
    ws.twB = base + o_twB;
    ws.tw4 = base + o_tw4;
    ws.deconv = base + o_deconv;
    ws.deconv_slot = base + o_deconv_slot;

    // The last-block counters and the status word must start at zero.
    cudaError_t e = cudaMemsetAsync(base + o_counter, 0, 256, st);
    if (e != cudaSuccess) return LS_ERR_CUDA;

    // Tables: roots of N2, N1 and n, then 1/phi_hat (nodes passed through scratch).
    k_root_table<T><<<64, 256, 0, st>>>(static_cast<T *>(ws.twA), n2, 6);
    k_root_table<T><<<64, 256, 0, st>>>(static_cast<T *>(ws.twB), n1, 6);
    k_root_table<T><<<256, 256, 0, st>>>(static_cast<T *>(ws.tw4), n, kTw4Bits);
    double quad[2 * kMaxQuad];
    const int q = es_quadrature_into(w, beta, quad, quad + kMaxQuad, kMaxQuad);
    if (q < 0) return LS_ERR_UNSUPPORTED;
    double *dquad = reinterpret_cast<double *>(base + o_quad);
    e = cudaMemcpyAsync(dquad, quad, sizeof(quad), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return LS_ERR_CUDA;
    e = launch_deconv_table<T>(g, ws.deconv, ndeconv, dquad, dquad + kMaxQuad, q, st);
    if (e != cudaSuccess) return LS_ERR_CUDA;
    e = launch_deconv_slot<T>(g, ws.deconv_slot, ws.deconv, ndeconv, st);
    if (e != cudaSuccess) return LS_ERR_CUDA;

    Batch bt;
    bt.S = 1;
    bt.many = nullptr;
    bt.one.pt_off = 0;
    bt.one.y_off = 0;
    bt.one.rec_off = 0;
    bt.one.nd = nd;
    bt.one.out_off = 0;
    bt.one.nf = nf;
    int neg;
    decompose_double(df, bt.one.ph.df_m, bt.one.ph.df_e, neg);
    decompose_double(f0, bt.one.ph.f0_m, bt.one.ph.f0_e, bt.one.ph.f0_neg);
    bt.one.ph.K0 = nf / 2;
    e = launch_pipeline<T>(g, ws, nd, bt, nd, t, y, dy, power, nullptr, nred, st, nullptr);
    if (e != cudaSuccess) return LS_ERR_CUDA;
    // Synchronous: wait (the host copy of the quadrature nodes also lives on
    // this stack frame) and read the device-side status.
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LS_ERR_CUDA;
    int h = 0;
    e = cudaMemcpy(&h, ws.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return LS_ERR_CUDA;
    if (h & kStatBadInput) return LS_ERR_ARG;
    if (h & kStatDegenerate) return LS_ERR_DEGENERATE;
    return LS_OK;
}

}  // namespace
}  // namespace nls

extern "C" ls_status ls_execute_noalloc(const double *t, const double *y, const double *dy,
                                        int64_t nd, double f0, double df, int64_t nf, double eps,
                                        int prec, double *power, void *stream)
{
    using namespace nls;
    if (!t || !y || !power) return LS_ERR_ARG;
    if (nd < 2 || nf < 1) return LS_ERR_ARG;
    if (!(df > 0.0) || !isfinite(df) || !isfinite(f0)) return LS_ERR_ARG;
    if (prec != LS_FP32 && prec != LS_FP64) return LS_ERR_ARG;
    if (nd > LS_NOALLOC_MAX_ND || nf > LS_NOALLOC_MAX_NF) return LS_ERR_UNSUPPORTED;
    if (!device_pointer(t) || !device_pointer(y) || !device_pointer(power) ||
        (dy && !device_pointer(dy)))
        return LS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LS_ERR_CUDA;
    unsigned char *base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return LS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return prec == LS_FP32
               ? run_noalloc<float>(base, t, y, dy, nd, f0, df, nf, eps, power, st)
               : run_noalloc<double>(base, t, y, dy, nd, f0, df, nf, eps, power, st);
}
