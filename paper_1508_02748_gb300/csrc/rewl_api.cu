// C ABI of librewl (include/rewl.h): window geometry, workspace layout,
// run orchestration (cycles of sample -> exchange -> check, replayed as CUDA
// graphs), state access and the final join.  Every arithmetic step of the
// method runs in the kernels of rewl_kernels.cu and rewl_join.cu; this file
// only sets up integer geometry and queues work.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "rewl_internal.cuh"

using namespace rewl;

struct rewl_s {
    rewl_config cfg;
    Params p;
    JoinScratch j;
    cudaStream_t stream;
    char err[512];
    unsigned long long host_cycle;   // cycles queued (equals the device count until done)
    int max_pairs;
    int wpb;
    int32_t *d_fail;
    uint8_t *d_stage;                // staging bytes (aliases the joined table)
    cudaGraphExec_t graph;           // check_every cycles, the last one checking
    bool graph_ok;
    int first_active;                // a walker of a non-empty window (-1 if none)
    double *jk_mean, *jk_err;        // jackknife results (device)
    std::vector<int> live;           // walkers of non-empty windows, in walker order
    // plain form: streams the per-walker launches are spread over, and one
    // event per stream plus one on the run's stream to fork and join them
    cudaStream_t plain_s[REWL_PLAIN_STREAMS];
    cudaEvent_t plain_ev[REWL_PLAIN_STREAMS + 1];
    bool plain_ok;
};

namespace {

const char *g_noerr = "";
char g_create_err[512];

int fail(rewl_t *h, int code, const char *fmt, ...)
{
    char *dst = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), REWL_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

namespace rewl {

// ----------------------------------------------------------- geometry ----

// Equal-sized overlapping windows over `bins` bins (Sec. 2, Fig. 1b; Sec. 3
// "equal-sized windows"): width ceil(bins / (1 + (n-1)(1-overlap))), the n
// starts spread evenly over [0, bins - width], rounded half up.
void axis_windows(int bins, int n, double overlap, std::vector<int> &lo, std::vector<int> &hi)
{
    lo.assign(n, 0);
    hi.assign(n, bins - 1);
    if (n == 1) return;
    const double denom = 1.0 + (double)(n - 1) * (1.0 - overlap);
    const double ratio = (double)bins / denom;
    long long width = (long long)std::ceil(ratio);
    if (width > bins) width = bins;
    if (width < 1) width = 1;
    const long long slack = bins - width;
    for (int k = 0; k < n; ++k) {
        const long long twice = 2LL * k * slack + (n - 1);   // round half up of k*slack/(n-1)
        lo[k] = (int)(twice / (2LL * (n - 1)));
        hi[k] = lo[k] + (int)width - 1;
    }
}

// A bin (e, m) can hold a configuration only if its broken-bond count
// b = 2e lies between the fewest bonds a minority of k = min(m, N-m) spins
// must break (compact droplet, 2 ceil(2 sqrt k), or a stripe wrapping the
// torus, 2L plus 2 when k is not a multiple of L) and the most it can break
// (4 per minority spin: b <= 2N - 2|2m - N|).  Sec. 1: the (E, M) plane has
// empty regions; windows inside them get no walkers.
bool bin_can_hold(int L, int e, int m)
{
    const int N = L * L;
    const int k = std::min(m, N - m);
    const int broken = 2 * e;
    if (broken > 2 * N - 2 * std::abs(2 * m - N)) return false;
    if (k == 0) return broken == 0;
    int c = (int)std::floor(2.0 * std::sqrt((double)k));
    while (c * c < 4 * k) ++c;                 // c = ceil(2 sqrt k), exactly
    while (c > 0 && (c - 1) * (c - 1) >= 4 * k) --c;
    const int droplet = 2 * c;
    const int stripe = 2 * L + (k % L ? 2 : 0);
    return broken >= std::min(droplet, stripe);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// x = 2^k for an integer k (x finite and positive)
bool is_pow2(double x)
{
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    int ex = 0;
    return std::frexp(x, &ex) == 0.5;
}

struct Layout {
    size_t st, rect, active, spins, we, wm, wt, wflat, lng, H, scr;
    size_t piece, off, GE, eshift, efrom, eto, ematch, rowok, F, mshift, mfrom, mto, mmatch, J, red, marg, gbuf;
    size_t eslice, mslice;
    size_t jk_ref, jk_sum, jk_sq, jk_mean, jk_err;
    size_t fail, total;
};

int check_config(const rewl_config *c, const char **why)
{
    if (!c) { *why = "null config"; return REWL_E_INVALID; }
    if (c->struct_size != sizeof(rewl_config)) { *why = "struct_size mismatch"; return REWL_E_INVALID; }
    if (c->L < 4 || c->L > 64) { *why = "L must be in [4, 64]"; return REWL_E_INVALID; }
    const int N = c->L * c->L;
    if (c->n_win_E < 1 || c->n_win_M < 1 || c->n_win_E > N + 1 || c->n_win_M > N + 1) { *why = "bad window grid"; return REWL_E_INVALID; }
    if (!(c->overlap_E >= 0.0 && c->overlap_E < 1.0 && c->overlap_M >= 0.0 && c->overlap_M < 1.0)) { *why = "overlap must be in [0, 1)"; return REWL_E_INVALID; }
    if (c->walkers_per_window < 1 || c->walkers_per_window > 1024) { *why = "walkers_per_window must be in [1, 1024]"; return REWL_E_INVALID; }
    if (c->precision != REWL_FP64 && c->precision != REWL_F32X2 && c->precision != REWL_F32) { *why = "unknown precision"; return REWL_E_INVALID; }
    if (!(c->lnf_init > 0.0 && c->lnf_final > 0.0 && c->lnf_factor > 0.0 && c->lnf_factor < 1.0)) { *why = "bad ln f schedule"; return REWL_E_INVALID; }
    if (!is_pow2(c->lnf_init) || !is_pow2(c->lnf_factor) || c->lnf_init < 0x1p-60) {
        *why = "lnf_init and lnf_factor must be powers of two (ln f = 2^-k keeps every ln g exact), lnf_init >= 2^-60";
        return REWL_E_INVALID;
    }
    if (!(c->flatness > 0.0 && c->flatness <= 1.0)) { *why = "flatness must be in (0, 1]"; return REWL_E_INVALID; }
    if (c->exchange_interval < 1) { *why = "exchange_interval must be >= 1"; return REWL_E_INVALID; }
    if (c->check_every < 1) { *why = "check_every must be >= 1"; return REWL_E_INVALID; }
    if (c->walkers_per_block < 0 || c->walkers_per_block > 128) { *why = "walkers_per_block must be in [0, 128]"; return REWL_E_INVALID; }
    if (c->sampler != REWL_SAMPLER_WARP && c->sampler != REWL_SAMPLER_THREAD) { *why = "unknown sampler"; return REWL_E_INVALID; }
    if (c->sampler == REWL_SAMPLER_WARP && c->walkers_per_block > 8) { *why = "warp sampler: walkers_per_block (warps per block) must be in [0, 8]"; return REWL_E_INVALID; }
    if (c->lanes_per_walker != 0 && c->lanes_per_walker != 8 && c->lanes_per_walker != 16 && c->lanes_per_walker != 32) { *why = "lanes_per_walker must be 0, 8, 16 or 32"; return REWL_E_INVALID; }
    if (c->table_mode < REWL_TABLES_AUTO || c->table_mode > REWL_TABLES_STAGED) { *why = "unknown table_mode"; return REWL_E_INVALID; }
    if (c->lattice_mode < REWL_LATTICE_AUTO || c->lattice_mode > REWL_LATTICE_SHARED) { *why = "unknown lattice_mode"; return REWL_E_INVALID; }
    if (c->lattice_mode == REWL_LATTICE_REGISTER && c->L * c->L > 64) { *why = "a register lattice needs N <= 64"; return REWL_E_INVALID; }
    return REWL_OK;
}

Dims dims_of(const rewl_config *c)
{
    Dims d;
    d.precision = c->precision;
    d.L = c->L; d.N = c->L * c->L;
    d.wpr = (c->L + 31) / 32;
    d.nwords = d.L * d.wpr;
    d.nE = c->n_win_E; d.nM = c->n_win_M; d.W = c->walkers_per_window;
    d.nwin = d.nE * d.nM; d.nwalk = d.nwin * d.W;
    std::vector<int> lo, hi;
    axis_windows(d.N + 1, d.nE, c->overlap_E, lo, hi);
    d.wE = hi[0] - lo[0] + 1;
    axis_windows(d.N + 1, d.nM, c->overlap_M, lo, hi);
    d.wM = hi[0] - lo[0] + 1;
    d.T = d.wE * d.wM;
    d.tstride = ((long long)d.T + 63) / 64 * 64;
    return d;
}

}  // namespace rewl

namespace {

Layout layout_of(const Dims &d)
{
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    const size_t B = (size_t)d.N + 1;
    L.st = take(sizeof(DevState));
    L.rect = take(sizeof(int4) * d.nwin);
    L.active = take(sizeof(int32_t) * d.nwin);
    L.spins = take(sizeof(uint32_t) * (size_t)d.nwords * d.nwalk);
    L.we = take(sizeof(int32_t) * d.nwalk);
    L.wm = take(sizeof(int32_t) * d.nwalk);
    L.wt = take(sizeof(unsigned long long) * d.nwalk);
    L.wflat = take(sizeof(int32_t) * d.nwalk);
    L.lng = take(8 * (size_t)d.nwalk * d.tstride);
    L.H = take(4 * (size_t)d.nwalk * d.tstride);
    L.scr = take(d.precision == REWL_F32 ? 0 : 4 * (size_t)d.nwalk * d.tstride);
    L.piece = take(8 * (size_t)d.nwin * d.tstride);
    L.off = take(8 * (size_t)d.nwalk);
    L.GE = take(8 * (size_t)d.nwin * d.wE);
    L.eshift = take(8 * (size_t)d.nwin);
    L.efrom = take(4 * (size_t)d.nwin);
    L.eto = take(4 * (size_t)d.nwin);
    L.ematch = take(4 * (size_t)d.nM * (d.nE > 1 ? d.nE - 1 : 1));
    L.rowok = take(4 * (size_t)d.nM);
    L.F = take(8 * (size_t)d.nM * B);
    L.mshift = take(8 * (size_t)d.nM);
    L.mfrom = take(4 * (size_t)d.nM);
    L.mto = take(4 * (size_t)d.nM);
    L.mmatch = take(4 * (size_t)(d.nM > 1 ? d.nM - 1 : 1));
    L.J = take(std::max(8 * B * B, (size_t)d.nwalk * d.N));
    L.red = take(8 * 2048);
    L.marg = take(8 * B);
    L.gbuf = take(8 * 2 * B * (size_t)d.nM);
    L.eslice = take(8 * (size_t)d.nwin * d.wM);
    L.mslice = take(8 * (size_t)d.nM * B);
    L.jk_ref = take(8 * B * B);
    L.jk_sum = take(8 * B * B);
    L.jk_sq = take(8 * B * B);
    L.jk_mean = take(8 * B * B);
    L.jk_err = take(8 * B * B);
    L.fail = take(4);
    L.total = o;
    return L;
}

int max_pairs_of(const Dims &d)
{
    int best = 0;
    for (int phase = 0; phase < 4; ++phase) {
        const int axis = phase >> 1, parity = phase & 1;
        const int nA = axis == 0 ? d.nE : d.nM, nO = axis == 0 ? d.nM : d.nE;
        const int per = (nA - parity) / 2;
        best = std::max(best, per > 0 ? per * nO : 0);
    }
    return best;
}

int sync(rewl_t *h)
{
    CK(h, cudaStreamSynchronize(h->stream));
    return REWL_OK;
}

int read_state(rewl_t *h, DevState *ds)
{
    CK(h, cudaMemcpyAsync(ds, h->p.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (ds->error & ERR_OVERFLOW) return fail(h, REWL_E_OVERFLOW, "histogram entry above INT32_MAX");
    return REWL_OK;
}

unsigned long long trials_of(rewl_t *h)
{
    unsigned long long t = 0;
    if (h->first_active < 0) return 0;
    if (cudaMemcpy(&t, h->p.wt + h->first_active, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
    return t;
}

void fill_status(rewl_t *h, const DevState &ds, rewl_status *s)
{
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
    s->iteration = ds.iter;
    s->done = ds.done;
    s->lnf = ds.lnf;
    s->cycles = ds.cycle;
    s->trials = trials_of(h);
    s->exch_attempts = ds.exch_attempts;
    s->exch_accepts = ds.exch_accepts;
    s->n_flat = ds.nflat_last;
    s->n_walkers = h->p.n_active_walkers;
    s->error = ds.error;
}

// One cycle's kernels: sample, exchange, [flat check], counters, [H reset].
cudaError_t queue_cycle(rewl_t *h, bool check)
{
    cudaError_t e;
    if ((e = launch_sweep(h->p, h->cfg.exchange_interval, h->wpb, h->stream)) != cudaSuccess) return e;
    if ((e = launch_exchange(h->p, h->max_pairs, h->stream)) != cudaSuccess) return e;
    if (check && (e = launch_flat(h->p, h->stream)) != cudaSuccess) return e;
    if ((e = launch_decide(h->p, DECIDE_XSTEP | DECIDE_CYCLE | (check ? DECIDE_CHECK : 0), h->stream)) != cudaSuccess) return e;
    if (check && (e = launch_fold(h->p, 1, h->stream)) != cudaSuccess) return e;
    return cudaSuccess;
}

int build_graph(rewl_t *h)
{
    if (h->graph_ok || h->stream == nullptr) return REWL_OK;
    cudaGraph_t g;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t qe = cudaSuccess;
    for (int c = 0; c < h->cfg.check_every && qe == cudaSuccess; ++c)
        qe = queue_cycle(h, c == h->cfg.check_every - 1);
    cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
    if (qe != cudaSuccess) return fail(h, REWL_E_CUDA, "queue during capture: %s", cudaGetErrorString(qe));
    if (ce != cudaSuccess) return fail(h, REWL_E_CUDA, "capture: %s", cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(h, REWL_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    h->graph_ok = true;
    return REWL_OK;
}

// Queues n cycles: whole check blocks through the graph, the rest eagerly.
int queue_cycles(rewl_t *h, unsigned long long n)
{
    const unsigned long long ce = (unsigned long long)h->cfg.check_every;
    while (n > 0) {
        if (h->host_cycle % ce == 0 && n >= ce && h->stream != nullptr) {
            int rc = build_graph(h);
            if (rc) return rc;
            CK(h, cudaGraphLaunch(h->graph, h->stream));
            h->host_cycle += ce;
            n -= ce;
        } else {
            const bool check = (h->host_cycle + 1) % ce == 0;
            CK(h, queue_cycle(h, check));
            h->host_cycle += 1;
            n -= 1;
        }
    }
    return REWL_OK;
}

}  // namespace

// ---------------------------------------------------------------- ABI ----

extern "C" int rewl_workspace_size(const rewl_config *cfg, size_t *bytes)
{
    const char *why = nullptr;
    int rc = check_config(cfg, &why);
    if (rc) return fail(nullptr, rc, "%s", why);
    if (!bytes) return fail(nullptr, REWL_E_INVALID, "null bytes");
    *bytes = layout_of(dims_of(cfg)).total;
    return REWL_OK;
}

namespace {

// Handle setup; `initialise` draws the spins and drives the walkers (a
// restored run gets its state from a checkpoint instead).
int create_impl(const rewl_config *cfg, const uint8_t *host_init_spins, void *d_workspace, size_t workspace_bytes,
                void *stream, rewl_t **out, bool initialise)
{
    const char *why = nullptr;
    int rc = check_config(cfg, &why);
    if (rc) return fail(nullptr, rc, "%s", why);
    if (!out || !d_workspace) return fail(nullptr, REWL_E_INVALID, "null output or workspace");
    if (((uintptr_t)d_workspace & 255u) != 0) return fail(nullptr, REWL_E_INVALID, "workspace not 256-byte aligned");
    const Dims d = dims_of(cfg);
    const Layout lay = layout_of(d);
    if (workspace_bytes < lay.total)
        return fail(nullptr, REWL_E_CAPACITY, "workspace %zu bytes < %zu needed", workspace_bytes, lay.total);

    rewl_t *h = new (std::nothrow) rewl_t();
    if (!h) return fail(nullptr, REWL_E_INVALID, "out of host memory");
    h->cfg = *cfg;
    h->stream = (cudaStream_t)stream;
    h->err[0] = 0;
    h->host_cycle = 0;
    h->wpb = cfg->walkers_per_block;
    h->graph_ok = false;
    h->max_pairs = max_pairs_of(d);

    char *base = (char *)d_workspace;
    Params &p = h->p;
    p.L = d.L; p.N = d.N; p.wpr = d.wpr; p.nwords = d.nwords;
    p.nE = d.nE; p.nM = d.nM; p.W = d.W; p.nwin = d.nwin; p.nwalk = d.nwalk;
    p.wE = d.wE; p.wM = d.wM; p.T = d.T; p.tstride = d.tstride;
    p.precision = cfg->precision;
    p.sampler = cfg->sampler;
    // stage the tables in shared memory when a warp's share stays small
    p.smt = 0;
    p.key0 = (uint32_t)cfg->seed; p.key1 = (uint32_t)(cfg->seed >> 32);
    p.divL = (uint32_t)((0x100000000ull + (unsigned long long)d.L - 1) / (unsigned long long)d.L);
    p.lnf_final = cfg->lnf_final; p.lnf_factor = cfg->lnf_factor;
    p.flat_q = (long long)std::llround(cfg->flatness * 1e6);
    p.drive_budget = cfg->drive_budget;
    p.join_exclude = -1;
    p.rect = (const int4 *)(base + lay.rect);
    p.active = (const int32_t *)(base + lay.active);
    p.spins = (uint32_t *)(base + lay.spins);
    p.we = (int32_t *)(base + lay.we);
    p.wm = (int32_t *)(base + lay.wm);
    p.wt = (unsigned long long *)(base + lay.wt);
    p.wflat = (int32_t *)(base + lay.wflat);
    p.lng = (double *)(base + lay.lng);
    p.lng2 = (float2 *)(base + lay.lng);
    p.lng1 = (float *)(base + lay.lng);
    p.H = (int32_t *)(base + lay.H);
    p.scr = (float *)(base + lay.scr);
    p.st = (DevState *)(base + lay.st);
    JoinScratch &j = h->j;
    j.piece = (double *)(base + lay.piece);
    j.off = (double *)(base + lay.off);
    j.GE = (double *)(base + lay.GE);
    j.eshift = (double *)(base + lay.eshift);
    j.efrom = (int32_t *)(base + lay.efrom);
    j.eto = (int32_t *)(base + lay.eto);
    j.ematch = (int32_t *)(base + lay.ematch);
    j.rowok = (int32_t *)(base + lay.rowok);
    j.F = (double *)(base + lay.F);
    j.mshift = (double *)(base + lay.mshift);
    j.mfrom = (int32_t *)(base + lay.mfrom);
    j.mto = (int32_t *)(base + lay.mto);
    j.mmatch = (int32_t *)(base + lay.mmatch);
    j.J = (double *)(base + lay.J);
    j.red = (double *)(base + lay.red);
    j.marg = (double *)(base + lay.marg);
    j.gbuf = (double *)(base + lay.gbuf);
    j.eslice = (double *)(base + lay.eslice);
    j.mslice = (double *)(base + lay.mslice);
    j.jk_ref = (double *)(base + lay.jk_ref);
    j.jk_sum = (double *)(base + lay.jk_sum);
    j.jk_sq = (double *)(base + lay.jk_sq);
    h->jk_mean = (double *)(base + lay.jk_mean);
    h->jk_err = (double *)(base + lay.jk_err);
    h->d_fail = (int32_t *)(base + lay.fail);
    h->d_stage = (uint8_t *)(base + lay.J);

    // Geometry on the host (integer setup), then uploaded.
    std::vector<int> elo, ehi, mlo, mhi;
    axis_windows(d.N + 1, d.nE, cfg->overlap_E, elo, ehi);
    axis_windows(d.N + 1, d.nM, cfg->overlap_M, mlo, mhi);
    std::vector<int4> rect(d.nwin);
    std::vector<int32_t> active(d.nwin, 0);
    int n_active = 0;
    for (int b = 0; b < d.nM; ++b)
        for (int a = 0; a < d.nE; ++a) {
            const int win = b * d.nE + a;
            rect[win] = make_int4(elo[a], ehi[a], mlo[b], mhi[b]);
            bool any = false;
            for (int e = elo[a]; e <= ehi[a] && !any; ++e)
                for (int m = mlo[b]; m <= mhi[b] && !any; ++m) any = bin_can_hold(d.L, e, m);
            active[win] = any ? 1 : 0;
            n_active += any ? 1 : 0;
        }
    p.n_active_walkers = n_active * d.W;
    // lanes per walker: a whole warp while walkers are few, packed groups when
    // the walkers alone can fill the GPU
    if (cfg->lanes_per_walker) p.group = cfg->lanes_per_walker;
    else p.group = p.n_active_walkers <= 1216 ? 32 : (p.n_active_walkers <= 2432 ? 16 : 8);
    p.lattice_reg = (cfg->lattice_mode == REWL_LATTICE_SHARED || d.N > 64 || d.wpr != 1) ? 0 : 1;
    // where the warp sampler keeps S and H during a launch: staged in shared
    // memory when a warp's share stays small, else global memory
    if (cfg->table_mode == REWL_TABLES_STAGED) p.smt = 1;
    else if (cfg->table_mode == REWL_TABLES_GLOBAL) p.smt = 0;
    else p.smt = tree_smem_per_warp(p, true) * (size_t)(32 / p.group) <= 100 * 1024 ? 1 : 0;
    if (p.sampler != REWL_SAMPLER_WARP) p.smt = 0;
    h->first_active = -1;
    for (int win = 0; win < d.nwin && h->first_active < 0; ++win)
        if (active[win]) h->first_active = win * d.W;
    for (int w = 0; w < d.nwalk; ++w)
        if (active[w / d.W]) h->live.push_back(w);

    auto bail = [&](int code) { rewl_destroy(h); return code; };
    DevState ds;
    std::memset(&ds, 0, sizeof(ds));
    ds.lnf = cfg->lnf_init;
    cudaError_t ce;
#define CKB(call)                                                                              \
    do {                                                                                       \
        ce = (call);                                                                           \
        if (ce != cudaSuccess) {                                                               \
            fail(nullptr, REWL_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(ce));        \
            return bail(REWL_E_CUDA);                                                          \
        }                                                                                      \
    } while (0)
    CKB(cudaMemcpyAsync(p.st, &ds, sizeof(ds), cudaMemcpyHostToDevice, h->stream));
    CKB(cudaMemcpyAsync((void *)p.rect, rect.data(), sizeof(int4) * d.nwin, cudaMemcpyHostToDevice, h->stream));
    CKB(cudaMemcpyAsync((void *)p.active, active.data(), sizeof(int32_t) * d.nwin, cudaMemcpyHostToDevice, h->stream));
    // Tables: ln g = 0, H = -1 (never visited).
    CKB(cudaMemsetAsync(p.lng, 0, 8 * (size_t)d.nwalk * d.tstride, h->stream));
    CKB(cudaMemsetAsync(p.H, 0xFF, 4 * (size_t)d.nwalk * d.tstride, h->stream));
    if (p.precision != REWL_F32) CKB(cudaMemsetAsync(p.scr, 0, 4 * (size_t)d.nwalk * d.tstride, h->stream));
    CKB(cudaMemsetAsync(h->d_fail, 0, 4, h->stream));
    if (!initialise) {
        CKB(cudaStreamSynchronize(h->stream));
        *out = h;
        return REWL_OK;
    }
    const uint8_t *d_bytes = nullptr;
    if (host_init_spins) {
        CKB(cudaMemcpyAsync(h->d_stage, host_init_spins, (size_t)d.nwalk * d.N, cudaMemcpyHostToDevice, h->stream));
        d_bytes = h->d_stage;
    }
    CKB(launch_init(p, d_bytes, h->stream));
    CKB(launch_drive(p, h->d_fail, h->stream));
    int32_t failed = 0;
    CKB(cudaMemcpyAsync(&failed, h->d_fail, 4, cudaMemcpyDeviceToHost, h->stream));
    CKB(cudaStreamSynchronize(h->stream));
#undef CKB
    if (failed) {
        fail(nullptr, REWL_E_UNREACHABLE, "a walker could not reach its window within %llu steps",
             (unsigned long long)cfg->drive_budget);
        return bail(REWL_E_UNREACHABLE);
    }
    *out = h;
    return REWL_OK;
}

}  // namespace

extern "C" int rewl_create(const rewl_config *cfg, const uint8_t *host_init_spins, void *d_workspace,
                           size_t workspace_bytes, void *stream, rewl_t **out)
{
    return create_impl(cfg, host_init_spins, d_workspace, workspace_bytes, stream, out, true);
}

// ------------------------------------------------------------- checkpoint ----

namespace {

const char kCkptMagic[8] = {'R', 'E', 'W', 'L', 'C', 'K', 'P', '2'};

struct CkptFile {
    FILE *f = nullptr;
    ~CkptFile() { if (f) fclose(f); }
};

// Device <-> file in chunks through one host buffer.
int dev_to_file(rewl_t *h, FILE *f, const void *dev, size_t bytes, std::vector<unsigned char> &buf)
{
    for (size_t o = 0; o < bytes; o += buf.size()) {
        const size_t n = std::min(buf.size(), bytes - o);
        CK(h, cudaMemcpyAsync(buf.data(), (const unsigned char *)dev + o, n, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (fwrite(buf.data(), 1, n, f) != n) return fail(h, REWL_E_INVALID, "checkpoint write failed");
    }
    return REWL_OK;
}

int file_to_dev(rewl_t *h, FILE *f, void *dev, size_t bytes, std::vector<unsigned char> &buf)
{
    for (size_t o = 0; o < bytes; o += buf.size()) {
        const size_t n = std::min(buf.size(), bytes - o);
        if (fread(buf.data(), 1, n, f) != n) return fail(h, REWL_E_INVALID, "checkpoint truncated");
        CK(h, cudaMemcpyAsync((unsigned char *)dev + o, buf.data(), n, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return REWL_OK;
}

struct StateRegion {
    void *dev;
    size_t bytes;
};

std::vector<StateRegion> state_regions(rewl_t *h)
{
    const Params &p = h->p;
    const size_t tab = (size_t)p.nwalk * (size_t)p.tstride;
    return {{p.st, sizeof(DevState)},
            {p.spins, 4 * (size_t)p.nwords * p.nwalk},
            {p.we, 4 * (size_t)p.nwalk},
            {p.wm, 4 * (size_t)p.nwalk},
            {p.wt, 8 * (size_t)p.nwalk},
            {p.wflat, 4 * (size_t)p.nwalk},
            {p.lng, 8 * tab},
            {p.H, 4 * tab}};
}

}  // namespace

extern "C" int rewl_save(rewl_t *h, const char *path)
{
    if (!h || !path) return REWL_E_INVALID;
    CK(h, cudaStreamSynchronize(h->stream));
    CkptFile cf;
    cf.f = fopen(path, "wb");
    if (!cf.f) return fail(h, REWL_E_INVALID, "cannot open %s for writing", path);
    const uint32_t version = 2, csize = (uint32_t)sizeof(rewl_config);
    const unsigned long long hc = h->host_cycle;
    if (fwrite(kCkptMagic, 1, 8, cf.f) != 8 || fwrite(&version, 4, 1, cf.f) != 1 || fwrite(&csize, 4, 1, cf.f) != 1 ||
        fwrite(&h->cfg, sizeof(rewl_config), 1, cf.f) != 1 || fwrite(&hc, 8, 1, cf.f) != 1)
        return fail(h, REWL_E_INVALID, "checkpoint write failed");
    std::vector<unsigned char> buf((size_t)64 << 20);
    for (const StateRegion &r : state_regions(h)) {
        const int rc = dev_to_file(h, cf.f, r.dev, r.bytes, buf);
        if (rc) return rc;
    }
    return REWL_OK;
}

extern "C" int rewl_checkpoint_config(const char *path, rewl_config *cfg)
{
    if (!path || !cfg) return fail(nullptr, REWL_E_INVALID, "null argument");
    CkptFile cf;
    cf.f = fopen(path, "rb");
    if (!cf.f) return fail(nullptr, REWL_E_INVALID, "cannot open %s", path);
    char magic[8];
    uint32_t version = 0, csize = 0;
    if (fread(magic, 1, 8, cf.f) != 8 || std::memcmp(magic, kCkptMagic, 8) != 0 || fread(&version, 4, 1, cf.f) != 1 ||
        fread(&csize, 4, 1, cf.f) != 1 || version != 2 || csize != sizeof(rewl_config) ||
        fread(cfg, sizeof(rewl_config), 1, cf.f) != 1)
        return fail(nullptr, REWL_E_INVALID, "%s is not a librewl checkpoint of this version", path);
    return REWL_OK;
}

extern "C" int rewl_load(const char *path, void *d_workspace, size_t workspace_bytes, void *stream, rewl_t **out)
{
    rewl_config cfg;
    int rc = rewl_checkpoint_config(path, &cfg);
    if (rc) return rc;
    CkptFile cf;
    cf.f = fopen(path, "rb");
    if (!cf.f) return fail(nullptr, REWL_E_INVALID, "cannot open %s", path);
    if (fseek(cf.f, 16 + (long)sizeof(rewl_config), SEEK_SET) != 0)
        return fail(nullptr, REWL_E_INVALID, "checkpoint truncated");
    unsigned long long hc = 0;
    if (fread(&hc, 8, 1, cf.f) != 1) return fail(nullptr, REWL_E_INVALID, "checkpoint truncated");
    rewl_t *h = nullptr;
    rc = create_impl(&cfg, nullptr, d_workspace, workspace_bytes, stream, &h, false);
    if (rc) return rc;
    std::vector<unsigned char> buf((size_t)64 << 20);
    for (const StateRegion &r : state_regions(h)) {
        rc = file_to_dev(h, cf.f, r.dev, r.bytes, buf);
        if (rc) {
            fail(nullptr, rc, "%s", h->err);
            rewl_destroy(h);
            return rc;
        }
    }
    // the screens are derived from the restored tables
    if (launch_fold(h->p, 0, h->stream) != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) {
        fail(nullptr, REWL_E_CUDA, "screen refresh after restore failed");
        rewl_destroy(h);
        return REWL_E_CUDA;
    }
    h->host_cycle = hc;
    *out = h;
    return REWL_OK;
}

extern "C" int rewl_run_cycles(rewl_t *h, uint64_t n_cycles, rewl_status *status)
{
    if (!h) return REWL_E_INVALID;
    int rc = queue_cycles(h, n_cycles);
    if (rc) return rc;
    DevState ds;
    rc = read_state(h, &ds);
    if (rc) return rc;
    fill_status(h, ds, status);
    return REWL_OK;
}

namespace {

// The plain form of a cycle's sampling: one single-thread launch per walker,
// round-robin over REWL_PLAIN_STREAMS streams forked from and joined back
// into the run's stream.
int queue_sample_plain(rewl_t *h)
{
    if (!h->plain_ok) {
        for (int i = 0; i < REWL_PLAIN_STREAMS; ++i)
            CK(h, cudaStreamCreateWithFlags(&h->plain_s[i], cudaStreamNonBlocking));
        for (int i = 0; i <= REWL_PLAIN_STREAMS; ++i)
            CK(h, cudaEventCreateWithFlags(&h->plain_ev[i], cudaEventDisableTiming));
        h->plain_ok = true;
    }
    CK(h, cudaEventRecord(h->plain_ev[REWL_PLAIN_STREAMS], h->stream));
    for (int i = 0; i < REWL_PLAIN_STREAMS; ++i) CK(h, cudaStreamWaitEvent(h->plain_s[i], h->plain_ev[REWL_PLAIN_STREAMS], 0));
    for (size_t k = 0; k < h->live.size(); ++k)
        CK(h, launch_sweep_walker(h->p, h->live[k], h->cfg.exchange_interval, h->plain_s[k % REWL_PLAIN_STREAMS]));
    for (int i = 0; i < REWL_PLAIN_STREAMS; ++i) {
        CK(h, cudaEventRecord(h->plain_ev[i], h->plain_s[i]));
        CK(h, cudaStreamWaitEvent(h->stream, h->plain_ev[i], 0));
    }
    return REWL_OK;
}

}  // namespace

extern "C" int rewl_enqueue_cycle(rewl_t *h, int parts)
{
    if (!h || parts < 1 || parts > 7 || ((parts & REWL_PART_SAMPLE) && (parts & REWL_PART_SAMPLE_PLAIN)))
        return fail(h, REWL_E_INVALID, "bad parts %d", parts);
    if (parts & REWL_PART_SAMPLE) CK(h, launch_sweep(h->p, h->cfg.exchange_interval, h->wpb, h->stream));
    if (parts & REWL_PART_SAMPLE_PLAIN) {
        const int rc = queue_sample_plain(h);
        if (rc) return rc;
    }
    if (parts & REWL_PART_REST) {
        const bool check = (h->host_cycle + 1) % (unsigned long long)h->cfg.check_every == 0;
        CK(h, launch_exchange(h->p, h->max_pairs, h->stream));
        if (check) CK(h, launch_flat(h->p, h->stream));
        CK(h, launch_decide(h->p, DECIDE_XSTEP | DECIDE_CYCLE | (check ? DECIDE_CHECK : 0), h->stream));
        if (check) CK(h, launch_fold(h->p, 1, h->stream));
        h->host_cycle += 1;
    }
    return REWL_OK;
}

extern "C" int rewl_run_cycles_plain(rewl_t *h, uint64_t n_cycles, rewl_status *status)
{
    if (!h) return REWL_E_INVALID;
    for (uint64_t c = 0; c < n_cycles; ++c) {
        const int rc = rewl_enqueue_cycle(h, REWL_PART_SAMPLE_PLAIN | REWL_PART_REST);
        if (rc) return rc;
    }
    DevState ds;
    int rc = read_state(h, &ds);
    if (rc) return rc;
    fill_status(h, ds, status);
    return REWL_OK;
}

extern "C" int rewl_run_iteration(rewl_t *h, uint64_t max_cycles, rewl_status *status)
{
    if (!h) return REWL_E_INVALID;
    DevState ds;
    int rc = read_state(h, &ds);
    if (rc) return rc;
    const int it0 = ds.iter;
    if (ds.done) { fill_status(h, ds, status); return REWL_OK; }
    uint64_t ran = 0;
    const uint64_t ce = (uint64_t)h->cfg.check_every;
    while (ran < max_cycles) {
        // up to the next check boundary
        uint64_t n = ce - (h->host_cycle % ce);
        if (n > max_cycles - ran) n = max_cycles - ran;
        rc = queue_cycles(h, n);
        if (rc) return rc;
        ran += n;
        rc = read_state(h, &ds);
        if (rc) return rc;
        if (ds.done || ds.iter != it0) { fill_status(h, ds, status); return REWL_OK; }
    }
    fill_status(h, ds, status);
    return fail(h, REWL_E_BUDGET, "no iteration ended within %llu cycles", (unsigned long long)max_cycles);
}

extern "C" int rewl_sweep(rewl_t *h, uint64_t n_trials)
{
    if (!h) return REWL_E_INVALID;
    CK(h, launch_sweep(h->p, n_trials, h->wpb, h->stream));
    DevState ds;
    return read_state(h, &ds);
}

extern "C" int rewl_exchange(rewl_t *h)
{
    if (!h) return REWL_E_INVALID;
    CK(h, launch_exchange(h->p, h->max_pairs, h->stream));
    CK(h, launch_decide(h->p, DECIDE_XSTEP, h->stream));
    return sync(h);
}

extern "C" int rewl_check(rewl_t *h, int32_t *all_flat)
{
    if (!h) return REWL_E_INVALID;
    CK(h, launch_flat(h->p, h->stream));
    CK(h, launch_decide(h->p, DECIDE_CHECK, h->stream));
    CK(h, launch_fold(h->p, 1, h->stream));
    DevState ds;
    int rc = read_state(h, &ds);
    if (rc) return rc;
    if (all_flat) *all_flat = ds.advanced;
    return REWL_OK;
}

extern "C" int rewl_get_status(rewl_t *h, rewl_status *status)
{
    if (!h || !status) return REWL_E_INVALID;
    DevState ds;
    int rc = read_state(h, &ds);
    if (rc) return rc;
    fill_status(h, ds, status);
    return REWL_OK;
}

extern "C" int rewl_get_windows(rewl_t *h, int32_t *host_out, size_t capacity)
{
    if (!h || !host_out) return REWL_E_INVALID;
    const int n = h->p.nwin;
    if (capacity < (size_t)n * 5) return fail(h, REWL_E_CAPACITY, "need %d entries", n * 5);
    std::vector<int4> rect(n);
    std::vector<int32_t> act(n);
    CK(h, cudaMemcpyAsync(rect.data(), h->p.rect, sizeof(int4) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(act.data(), h->p.active, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < n; ++k) {
        host_out[5 * k + 0] = rect[k].x; host_out[5 * k + 1] = rect[k].y;
        host_out[5 * k + 2] = rect[k].z; host_out[5 * k + 3] = rect[k].w;
        host_out[5 * k + 4] = act[k];
    }
    return REWL_OK;
}

extern "C" int rewl_get_walkers(rewl_t *h, int64_t *host_state, uint8_t *host_spins)
{
    if (!h) return REWL_E_INVALID;
    const Params &p = h->p;
    std::vector<int32_t> e(p.nwalk), m(p.nwalk), f(p.nwalk);
    std::vector<unsigned long long> t(p.nwalk);
    CK(h, cudaMemcpyAsync(e.data(), p.we, 4 * (size_t)p.nwalk, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(m.data(), p.wm, 4 * (size_t)p.nwalk, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(f.data(), p.wflat, 4 * (size_t)p.nwalk, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(t.data(), p.wt, 8 * (size_t)p.nwalk, cudaMemcpyDeviceToHost, h->stream));
    std::vector<uint32_t> words;
    if (host_spins) {
        words.resize((size_t)p.nwords * p.nwalk);
        CK(h, cudaMemcpyAsync(words.data(), p.spins, 4 * words.size(), cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    for (int w = 0; w < p.nwalk; ++w) {
        if (host_state) {
            host_state[4 * w + 0] = e[w]; host_state[4 * w + 1] = m[w];
            host_state[4 * w + 2] = (int64_t)t[w]; host_state[4 * w + 3] = f[w];
        }
        if (host_spins)
            for (int i = 0; i < p.L; ++i)
                for (int jj = 0; jj < p.L; ++jj) {
                    const uint32_t wd = words[(size_t)(i * p.wpr + (jj >> 5)) * p.nwalk + w];
                    host_spins[(size_t)w * p.N + i * p.L + jj] = (uint8_t)((wd >> (jj & 31)) & 1u);
                }
    }
    return REWL_OK;
}

// Host copies of the tables.  Exact formats store base and H; the value
// handed out is ln g = base + max(H, 0) ln f, the sum formed in double (exact
// for the dyadic schedule), and rewl_set_tables stores base = ln g -
// max(H, 0) ln f and refreshes the screens on the device.
extern "C" int rewl_get_tables(rewl_t *h, double *host_lng, int32_t *host_H, size_t capacity)
{
    if (!h) return REWL_E_INVALID;
    const Params &p = h->p;
    const size_t n = (size_t)p.nwalk * p.T;
    if (capacity < n) return fail(h, REWL_E_CAPACITY, "need %zu entries", n);
    DevState ds;
    int rc = read_state(h, &ds);
    if (rc && rc != REWL_E_OVERFLOW) return rc;
    std::vector<int32_t> Hv(n);
    CK(h, cudaMemcpy2DAsync(Hv.data(), 4 * (size_t)p.T, p.H, 4 * (size_t)p.tstride, 4 * (size_t)p.T, p.nwalk,
                            cudaMemcpyDeviceToHost, h->stream));
    if (host_lng) {
        if (p.precision == REWL_FP64) {
            CK(h, cudaMemcpy2DAsync(host_lng, 8 * (size_t)p.T, p.lng, 8 * (size_t)p.tstride, 8 * (size_t)p.T,
                                    p.nwalk, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        } else if (p.precision == REWL_F32X2) {
            std::vector<float2> tmp(n);
            CK(h, cudaMemcpy2DAsync(tmp.data(), 8 * (size_t)p.T, p.lng2, 8 * (size_t)p.tstride, 8 * (size_t)p.T,
                                    p.nwalk, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            for (size_t i = 0; i < n; ++i) host_lng[i] = (double)tmp[i].x + (double)tmp[i].y;
        } else {
            std::vector<float> tmp(n);
            CK(h, cudaMemcpy2DAsync(tmp.data(), 4 * (size_t)p.T, p.lng1, 4 * (size_t)p.tstride, 4 * (size_t)p.T,
                                    p.nwalk, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            for (size_t i = 0; i < n; ++i) host_lng[i] = (double)tmp[i];
        }
        if (p.precision != REWL_F32)
            for (size_t i = 0; i < n; ++i)
                if (Hv[i] > 0) host_lng[i] += (double)Hv[i] * ds.lnf;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (host_H) std::memcpy(host_H, Hv.data(), 4 * n);
    return REWL_OK;
}

extern "C" int rewl_set_tables(rewl_t *h, const double *host_lng, const int32_t *host_H, size_t count)
{
    if (!h) return REWL_E_INVALID;
    const Params &p = h->p;
    const size_t n = (size_t)p.nwalk * p.T;
    if (count != n) return fail(h, REWL_E_CAPACITY, "need exactly %zu entries", n);
    DevState ds;
    int rc = read_state(h, &ds);
    if (rc && rc != REWL_E_OVERFLOW) return rc;
    std::vector<int32_t> Hv(n);
    if (host_H) {
        std::memcpy(Hv.data(), host_H, 4 * n);
    } else {
        CK(h, cudaMemcpy2DAsync(Hv.data(), 4 * (size_t)p.T, p.H, 4 * (size_t)p.tstride, 4 * (size_t)p.T, p.nwalk,
                                cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    if (host_lng) {
        std::vector<double> base(host_lng, host_lng + n);
        if (p.precision != REWL_F32)
            for (size_t i = 0; i < n; ++i)
                if (Hv[i] > 0) base[i] -= (double)Hv[i] * ds.lnf;
        if (p.precision == REWL_FP64) {
            CK(h, cudaMemcpy2DAsync(p.lng, 8 * (size_t)p.tstride, base.data(), 8 * (size_t)p.T, 8 * (size_t)p.T,
                                    p.nwalk, cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        } else if (p.precision == REWL_F32X2) {
            std::vector<float2> tmp(n);
            for (size_t i = 0; i < n; ++i) {
                const float hi = (float)base[i];
                tmp[i] = make_float2(hi, (float)(base[i] - (double)hi));
            }
            CK(h, cudaMemcpy2DAsync(p.lng2, 8 * (size_t)p.tstride, tmp.data(), 8 * (size_t)p.T, 8 * (size_t)p.T,
                                    p.nwalk, cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        } else {
            std::vector<float> tmp(n);
            for (size_t i = 0; i < n; ++i) tmp[i] = (float)base[i];
            CK(h, cudaMemcpy2DAsync(p.lng1, 4 * (size_t)p.tstride, tmp.data(), 4 * (size_t)p.T, 4 * (size_t)p.T,
                                    p.nwalk, cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        }
    }
    if (host_H)
        CK(h, cudaMemcpy2DAsync(p.H, 4 * (size_t)p.tstride, host_H, 4 * (size_t)p.T, 4 * (size_t)p.T, p.nwalk,
                                cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_fold(p, 0, h->stream));
    return sync(h);
}

extern "C" int rewl_tables_digest(rewl_t *h, uint64_t *digest)
{
    if (!h || !digest) return REWL_E_INVALID;
    unsigned long long *d = (unsigned long long *)h->d_stage;   // the staging area is free between calls
    CK(h, cudaMemsetAsync(d, 0, 8, h->stream));
    CK(h, launch_digest(h->p, d, h->stream));
    unsigned long long v = 0;
    CK(h, cudaMemcpyAsync(&v, d, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *digest = v;
    return REWL_OK;
}

extern "C" int rewl_get_lng(rewl_t *h, int what, double *host_out, size_t capacity, size_t *needed,
                            int32_t *host_ematch, int32_t *host_mmatch)
{
    if (!h) return REWL_E_INVALID;
    Params p = h->p;
    p.join_rule = (what & REWL_JOIN_PER_SLICE) ? 1 : 0;
    what &= ~REWL_JOIN_PER_SLICE;
    const size_t B = (size_t)p.N + 1;
    size_t n;
    if (what == REWL_LNG_JOINED) n = B * B;
    else if (what == REWL_LNG_MARGINAL_E) n = B;
    else return fail(h, REWL_E_INVALID, "unknown output kind %d", what);
    if (needed) *needed = n;
    if (!host_out || capacity < n) return fail(h, REWL_E_CAPACITY, "need %zu entries", n);
    CK(h, cudaMemsetAsync(&p.st->join_error, 0, sizeof(int32_t), h->stream));
    CK(h, launch_join(p, h->j, h->stream));
    if (what == REWL_LNG_MARGINAL_E) CK(h, launch_marginal_e(p, h->j, h->stream));
    DevState ds;
    int rc = read_state(h, &ds);
    if (rc) return rc;
    if (ds.join_error) return fail(h, REWL_E_JOIN, "join failed (code %d): adjacent pieces share no visited bins", ds.join_error);
    CK(h, cudaMemcpyAsync(host_out, what == REWL_LNG_JOINED ? h->j.J : h->j.marg, 8 * n, cudaMemcpyDeviceToHost, h->stream));
    if (host_ematch)
        CK(h, cudaMemcpyAsync(host_ematch, h->j.ematch, 4 * (size_t)p.nM * (p.nE > 1 ? p.nE - 1 : 1),
                              cudaMemcpyDeviceToHost, h->stream));
    if (host_mmatch)
        CK(h, cudaMemcpyAsync(host_mmatch, h->j.mmatch, 4 * (size_t)(p.nM > 1 ? p.nM - 1 : 1),
                              cudaMemcpyDeviceToHost, h->stream));
    return sync(h);
}

extern "C" int rewl_get_lng_jackknife(rewl_t *h, int what, double *host_mean, double *host_err, size_t capacity,
                                      size_t *needed)
{
    if (!h) return REWL_E_INVALID;
    Params p0 = h->p;
    p0.join_rule = (what & REWL_JOIN_PER_SLICE) ? 1 : 0;
    what &= ~REWL_JOIN_PER_SLICE;
    const size_t B = (size_t)p0.N + 1;
    size_t n;
    if (what == REWL_LNG_JOINED) n = B * B;
    else if (what == REWL_LNG_MARGINAL_E) n = B;
    else return fail(h, REWL_E_INVALID, "unknown output kind %d", what);
    if (needed) *needed = n;
    if (p0.W < 2) return fail(h, REWL_E_INVALID, "the jackknife needs at least two walkers per window");
    if (!host_mean || !host_err || capacity < n) return fail(h, REWL_E_CAPACITY, "need %zu entries", n);
    Params p = p0;
    for (int k = 0; k < p.W; ++k) {
        p.join_exclude = k;
        CK(h, cudaMemsetAsync(&p.st->join_error, 0, sizeof(int32_t), h->stream));
        CK(h, launch_join(p, h->j, h->stream));
        if (what == REWL_LNG_MARGINAL_E) CK(h, launch_marginal_e(p, h->j, h->stream));
        CK(h, launch_jk_accum(h->j, what == REWL_LNG_JOINED ? h->j.J : h->j.marg, n, k, h->stream));
        DevState ds;
        const int rc = read_state(h, &ds);
        if (rc) return rc;
        if (ds.join_error) return fail(h, REWL_E_JOIN, "jackknife replicate %d: join failed (code %d)", k, ds.join_error);
    }
    CK(h, launch_jk_final(h->j, h->jk_mean, h->jk_err, n, p.W, h->stream));
    CK(h, cudaMemcpyAsync(host_mean, h->jk_mean, 8 * n, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(host_err, h->jk_err, 8 * n, cudaMemcpyDeviceToHost, h->stream));
    return sync(h);
}

extern "C" const char *rewl_last_error(const rewl_t *h)
{
    if (!h) return g_create_err[0] ? g_create_err : g_noerr;
    return h->err;
}

extern "C" int rewl_destroy(rewl_t *h)
{
    if (!h) return REWL_OK;
    if (h->graph_ok) cudaGraphExecDestroy(h->graph);
    if (h->plain_ok) {
        for (int i = 0; i < REWL_PLAIN_STREAMS; ++i) cudaStreamDestroy(h->plain_s[i]);
        for (int i = 0; i <= REWL_PLAIN_STREAMS; ++i) cudaEventDestroy(h->plain_ev[i]);
    }
    delete h;
    return REWL_OK;
}

extern "C" int rewl_relative_difference(const double *d_lng_a, const double *d_lng_b, double *d_out, uint64_t n,
                                        void *stream)
{
    if (n && (!d_lng_a || !d_lng_b || !d_out)) return fail(nullptr, REWL_E_INVALID, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_rel_diff(d_lng_a, d_lng_b, d_out, (size_t)n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, REWL_E_CUDA, "relative difference: %s", cudaGetErrorString(e));
    return REWL_OK;
}

extern "C" int rewl_philox(const uint32_t *d_ctr, const uint32_t *key, uint32_t *d_out, uint64_t n, void *stream)
{
    if (!key || (n && (!d_ctr || !d_out))) return fail(nullptr, REWL_E_INVALID, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_philox(d_ctr, key[0], key[1], d_out, n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, REWL_E_CUDA, "philox: %s", cudaGetErrorString(e));
    return REWL_OK;
}

// ------------------------------------------------------------------ batch ----

struct rewl_batch_s {
    std::vector<rewl_t *> runs;
    std::vector<cudaStream_t> streams;   // one per run, created by the batch
    std::vector<cudaEvent_t> events;     // fork event + one join event per run
    cudaStream_t stream;
    cudaGraphExec_t graph;
    unsigned long long k;                // cycles per graph launch
    char err[512];
};

namespace {

unsigned long long gcd_u(unsigned long long a, unsigned long long b)
{
    while (b) { const unsigned long long t = a % b; a = b; b = t; }
    return a;
}

void batch_free(rewl_batch_t *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    delete b;
}

}  // namespace

extern "C" int rewl_batch_create(rewl_t *const *runs, int n, void *stream, rewl_batch_t **out)
{
    if (!runs || n < 1 || !out || !stream) return fail(nullptr, REWL_E_INVALID, "batch: bad arguments");
    rewl_batch_t *b = new (std::nothrow) rewl_batch_t();
    if (!b) return fail(nullptr, REWL_E_INVALID, "out of host memory");
    b->stream = (cudaStream_t)stream;
    b->graph = nullptr;
    b->k = 1;
    for (int i = 0; i < n; ++i) {
        rewl_t *h = runs[i];
        if (!h) { batch_free(b); return fail(nullptr, REWL_E_INVALID, "batch: null run %d", i); }
        const unsigned long long ce = (unsigned long long)h->cfg.check_every;
        if (h->host_cycle % ce != 0) {
            batch_free(b);
            return fail(nullptr, REWL_E_INVALID, "batch: run %d is not at a multiple of its check_every", i);
        }
        b->k = b->k / gcd_u(b->k, ce) * ce;
        if (b->k > 64) { batch_free(b); return fail(nullptr, REWL_E_INVALID, "batch: lcm of check_every above 64"); }
        b->runs.push_back(h);
    }
    cudaError_t e;
    b->events.resize(n + 1, nullptr);
    b->streams.resize(n, nullptr);
    for (int i = 0; i <= n; ++i)
        if ((e = cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming)) != cudaSuccess) {
            batch_free(b);
            return fail(nullptr, REWL_E_CUDA, "batch: event: %s", cudaGetErrorString(e));
        }
    for (int i = 0; i < n; ++i)
        if ((e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking)) != cudaSuccess) {
            batch_free(b);
            return fail(nullptr, REWL_E_CUDA, "batch: stream: %s", cudaGetErrorString(e));
        }
    // Capture: fork from the batch stream, K cycles of each run on its own
    // stream, join back.  The runs' own streams are swapped for the capture.
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        batch_free(b);
        return fail(nullptr, REWL_E_CUDA, "batch: begin capture: %s", cudaGetErrorString(e));
    }
    cudaError_t qe = cudaEventRecord(b->events[n], b->stream);
    for (int i = 0; i < n && qe == cudaSuccess; ++i) {
        rewl_t *h = b->runs[i];
        cudaStream_t own = h->stream;
        h->stream = b->streams[i];
        qe = cudaStreamWaitEvent(h->stream, b->events[n], 0);
        const unsigned long long ce = (unsigned long long)h->cfg.check_every;
        for (unsigned long long c = 0; c < b->k && qe == cudaSuccess; ++c)
            qe = queue_cycle(h, (c + 1) % ce == 0);
        if (qe == cudaSuccess) qe = cudaEventRecord(b->events[i], h->stream);
        if (qe == cudaSuccess) qe = cudaStreamWaitEvent(b->stream, b->events[i], 0);
        h->stream = own;
    }
    e = cudaStreamEndCapture(b->stream, &g);
    if (qe != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        batch_free(b);
        return fail(nullptr, REWL_E_CUDA, "batch: capture: %s",
                    cudaGetErrorString(qe != cudaSuccess ? qe : e));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        batch_free(b);
        return fail(nullptr, REWL_E_CUDA, "batch: instantiate: %s", cudaGetErrorString(e));
    }
    *out = b;
    return REWL_OK;
}

extern "C" int rewl_batch_cycles_per_launch(const rewl_batch_t *b, uint64_t *k)
{
    if (!b || !k) return REWL_E_INVALID;
    *k = b->k;
    return REWL_OK;
}

extern "C" int rewl_batch_run_cycles(rewl_batch_t *b, uint64_t n_cycles)
{
    if (!b) return REWL_E_INVALID;
    if (n_cycles % b->k != 0) return REWL_E_INVALID;
    for (uint64_t c = 0; c < n_cycles; c += b->k) {
        const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) return fail(nullptr, REWL_E_CUDA, "batch launch: %s", cudaGetErrorString(e));
    }
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(nullptr, REWL_E_CUDA, "batch sync: %s", cudaGetErrorString(e));
    for (rewl_t *h : b->runs) h->host_cycle += n_cycles;
    for (rewl_t *h : b->runs) {
        DevState ds;
        const int rc = read_state(h, &ds);
        if (rc) return rc;
    }
    return REWL_OK;
}

extern "C" int rewl_batch_enqueue(rewl_batch_t *b)
{
    if (!b) return REWL_E_INVALID;
    const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return fail(nullptr, REWL_E_CUDA, "batch launch: %s", cudaGetErrorString(e));
    for (rewl_t *h : b->runs) h->host_cycle += b->k;
    return REWL_OK;
}

extern "C" int rewl_batch_destroy(rewl_batch_t *b)
{
    batch_free(b);
    return REWL_OK;
}
