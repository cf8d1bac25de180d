// rewl_join_noalloc: the final merge / join / normalisation of librewl for
// callers that cannot allocate device memory.
//
// Who needs it: callers that may not call cudaMalloc -- a process whose
// device memory is all owned by an external allocator (a framework's caching
// pool), or one whose memory budget is fixed up front.  Such a caller still
// owns its inputs and output; what it cannot provide is the join's working
// memory.  This entry point takes that working memory from one file-scope
// device array of fixed size, so it calls no allocator at all.  It reads its
// error word back and synchronises on the caller's stream before returning.
//
// The array: kScratchBytes (8 MiB) of __device__ memory, present
// on every GPU that loads the library until the process exits.  Its device
// address is looked up once per device (cudaGetSymbolAddress, with that
// device current) by the first call made on that device; make that first call
// before any stream capture.  Every call shares the array and it keeps the
// last call's contents; everything a call reads from it is first written by
// the same call (the error word is cleared).  Calls that overlap on the GPU
// (two streams, or two host threads) race on the array and must be
// serialised by the caller.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "rewl_internal.cuh"

namespace rewl {

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_join_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};
thread_local char g_msg[512];    // message of this thread's last call

int say(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return code;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

}  // namespace rewl

using namespace rewl;

// The calling thread's last message (each host thread has its own).
extern "C" const char *rewl_noalloc_last_error(void) { return g_msg; }

extern "C" int rewl_join_noalloc(const rewl_config *cfg, const double *d_lng, const int32_t *d_H, double *d_out,
                                 void *stream)
{
    const char *why = nullptr;
    int rc = check_config(cfg, &why);
    if (rc) return say(rc, "%s", why);
    if (!d_lng || !d_H || !d_out) return say(REWL_E_INVALID, "null device pointer");
    const Dims d = dims_of(cfg);
    const size_t B = (size_t)d.N + 1;

    // Scratch layout (the join's working set for this geometry).
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = up256(o + bytes); return at; };
    const size_t o_st = take(sizeof(DevState));
    const size_t o_rect = take(sizeof(int4) * d.nwin);
    const size_t o_act = take(sizeof(int32_t) * d.nwin);
    const size_t o_piece = take(8 * (size_t)d.nwin * d.T);
    const size_t o_off = take(8 * (size_t)d.nwalk);
    const size_t o_GE = take(8 * (size_t)d.nwin * d.wE);
    const size_t o_eshift = take(8 * (size_t)d.nwin);
    const size_t o_efrom = take(4 * (size_t)d.nwin);
    const size_t o_eto = take(4 * (size_t)d.nwin);
    const size_t o_ematch = take(4 * (size_t)d.nM * (d.nE > 1 ? d.nE - 1 : 1));
    const size_t o_rowok = take(4 * (size_t)d.nM);
    const size_t o_F = take(8 * (size_t)d.nM * B);
    const size_t o_mshift = take(8 * (size_t)d.nM);
    const size_t o_mfrom = take(4 * (size_t)d.nM);
    const size_t o_mto = take(4 * (size_t)d.nM);
    const size_t o_mmatch = take(4 * (size_t)(d.nM > 1 ? d.nM - 1 : 1));
    const size_t o_red = take(8 * 2048);
    const size_t o_marg = take(8 * B);
    const size_t o_gbuf = take(8 * 2 * B * (size_t)d.nM);
    if (o > kScratchBytes)
        return say(REWL_E_CAPACITY,
                   "rewl_join_noalloc: this geometry needs %zu bytes of join scratch, above the fixed %zu "
                   "(L=%d, %dx%d windows of %d bins, %d walkers); use rewl_get_lng",
                   o, kScratchBytes, d.L, d.nE, d.nM, d.T, d.nwalk);

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return say(REWL_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
    if (dev < 0 || dev >= kMaxDevices) return say(REWL_E_INVALID, "device %d out of range", dev);
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            ce = cudaGetSymbolAddress(&ptr, g_join_scratch);
            if (ce != cudaSuccess) return say(REWL_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(ce));
            g_scratch_addr[dev] = (unsigned char *)ptr;
        }
        base = g_scratch_addr[dev];
    }

    // Geometry of the run the tables belong to (same rules as rewl_create).
    std::vector<int> elo, ehi, mlo, mhi;
    axis_windows(d.N + 1, d.nE, cfg->overlap_E, elo, ehi);
    axis_windows(d.N + 1, d.nM, cfg->overlap_M, mlo, mhi);
    std::vector<int4> rect(d.nwin);
    std::vector<int32_t> active(d.nwin, 0);
    for (int b = 0; b < d.nM; ++b)
        for (int a = 0; a < d.nE; ++a) {
            const int win = b * d.nE + a;
            rect[win] = make_int4(elo[a], ehi[a], mlo[b], mhi[b]);
            bool any = false;
            for (int e = elo[a]; e <= ehi[a] && !any; ++e)
                for (int m = mlo[b]; m <= mhi[b] && !any; ++m) any = bin_can_hold(d.L, e, m);
            active[win] = any ? 1 : 0;
        }

    Params p;
    std::memset(&p, 0, sizeof p);
    p.L = d.L; p.N = d.N; p.wpr = d.wpr; p.nwords = d.nwords;
    p.nE = d.nE; p.nM = d.nM; p.W = d.W; p.nwin = d.nwin; p.nwalk = d.nwalk;
    p.wE = d.wE; p.wM = d.wM; p.T = d.T;
    p.tstride = d.T;                         // caller tables: no padding between walkers
    p.precision = REWL_FP64;
    p.join_exclude = -1;                     // every walker takes part in the merge
    p.rect = (const int4 *)(base + o_rect);
    p.active = (const int32_t *)(base + o_act);
    p.lng = const_cast<double *>(d_lng);
    p.H = const_cast<int32_t *>(d_H);
    p.st = (DevState *)(base + o_st);
    JoinScratch j;
    std::memset(&j, 0, sizeof j);            // rule-1 and jackknife buffers stay unused (null)
    j.piece = (double *)(base + o_piece);
    j.off = (double *)(base + o_off);
    j.GE = (double *)(base + o_GE);
    j.eshift = (double *)(base + o_eshift);
    j.efrom = (int32_t *)(base + o_efrom);
    j.eto = (int32_t *)(base + o_eto);
    j.ematch = (int32_t *)(base + o_ematch);
    j.rowok = (int32_t *)(base + o_rowok);
    j.F = (double *)(base + o_F);
    j.mshift = (double *)(base + o_mshift);
    j.mfrom = (int32_t *)(base + o_mfrom);
    j.mto = (int32_t *)(base + o_mto);
    j.mmatch = (int32_t *)(base + o_mmatch);
    j.J = d_out;                             // the joined table is built in the caller's output
    j.red = (double *)(base + o_red);
    j.marg = (double *)(base + o_marg);
    j.gbuf = (double *)(base + o_gbuf);

    cudaStream_t s = (cudaStream_t)stream;
    // a zeroed state has ln f = 0: the join reads the caller's ln g as it is
    if ((ce = cudaMemsetAsync(p.st, 0, sizeof(DevState), s)) != cudaSuccess ||
        (ce = cudaMemcpyAsync((void *)p.rect, rect.data(), sizeof(int4) * d.nwin, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (ce = cudaMemcpyAsync((void *)p.active, active.data(), sizeof(int32_t) * d.nwin, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (ce = launch_join(p, j, s)) != cudaSuccess)
        return say(REWL_E_CUDA, "rewl_join_noalloc: %s", cudaGetErrorString(ce));
    int32_t jerr = 0;
    if ((ce = cudaMemcpyAsync(&jerr, &p.st->join_error, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (ce = cudaStreamSynchronize(s)) != cudaSuccess)
        return say(REWL_E_CUDA, "rewl_join_noalloc: %s", cudaGetErrorString(ce));
    if (jerr) return say(REWL_E_JOIN, "rewl_join_noalloc: join failed (code %d)", jerr);
    g_msg[0] = 0;
    return REWL_OK;
}
