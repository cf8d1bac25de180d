// Internal declarations of librewl (device path of two-dimensional
// replica-exchange Wang-Landau sampling, arXiv:1508.02748).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "rewl.h"

namespace rewl {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): two 32x32->64 products
// per round on counter words 0 and 2, high halves folded into the other words
// with the round key, key advanced by the two Weyl increments, ten rounds.
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = 0xD2511F53u * c0, ah = __umulhi(0xD2511F53u, c0);
        const uint32_t b = 0xCD9E8D57u * c2, bh = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = bh ^ c1 ^ k0;
        const uint32_t n2 = ah ^ c3 ^ k1;
        c0 = n0; c1 = b; c2 = n2; c3 = a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Stream tags of the counter's last word (one per kind of draw).
enum : uint32_t { TAG_INIT = 1, TAG_DRIVE = 2, TAG_TRIAL = 3, TAG_PERM = 4, TAG_EXCH = 5 };

// Scalars of a run that live in device memory (part of the workspace).
struct DevState {
    double lnf;                       // ln f of the current iteration
    double lnf_done;                  // ln f of the iteration that ended at the last advance
    unsigned long long cycle;         // cycles run
    unsigned long long xstep;         // exchange sweeps run (phase = xstep mod 4)
    unsigned long long exch_attempts;
    unsigned long long exch_accepts;
    int32_t iter;                     // completed iterations
    int32_t done;                     // final iteration flat
    int32_t nflat;                    // walkers found flat by the running check
    int32_t nflat_last;               // result of the last check
    int32_t advanced;                 // the last check ended an iteration
    int32_t error;                    // device error bits (ERR_*)
    int32_t join_error;
    int32_t pad;
};

enum : int32_t { ERR_OVERFLOW = 1, ERR_UNREACHABLE = 2 };

// Everything a kernel needs, passed by value.
struct Params {
    int L, N;
    int wpr;          // 32-bit words per lattice row
    int nwords;       // words per lattice = L * wpr
    int nE, nM, W;    // window grid, walkers per window
    int nwin, nwalk;
    int wE, wM;       // window extent in e and m (all windows equal)
    int T;            // bins per window = wE * wM
    long long tstride;// table entries per walker (T rounded up to 64)
    int n_active_walkers;
    int precision;
    int sampler;      // REWL_SAMPLER_WARP or REWL_SAMPLER_THREAD
    int smt;          // warp sampler: tables staged in shared memory
    int group;        // warp sampler: lanes per walker
    int lattice_reg;  // warp sampler: the lattice in a 64-bit register (N <= 64)
    uint32_t key0, key1;
    uint32_t divL;    // ceil(2^32 / L): site / L = umulhi(site, divL) for site < N
    double lnf_final, lnf_factor;
    long long flat_q; // round(flatness * 1e6)
    uint64_t drive_budget;

    int join_exclude; // merge: walker index within each window left out (-1: none)
    int join_rule;    // join steps: 0 one constant per piece, 1 one per slice (rewl.h REWL_JOIN_PER_SLICE)
    int walker0;      // thread sampler: walker of thread 0 of block 0 (0 for a whole sweep)

    const int4 *rect;       // per window: e0, e1, m0, m1
    const int32_t *active;  // per window: 1 if it can hold a configuration

    uint32_t *spins;  // nwords x nwalk, word-major: word k of walker w at k * nwalk + w
    int32_t *we, *wm; // bins of each walker's configuration
    unsigned long long *wt;  // trials done per walker
    int32_t *wflat;   // last flatness verdict
    // Tables, nwalk x tstride entries each.  Exact formats (REWL_FP64,
    // REWL_F32X2) hold ln g(b) = base(b) + max(H(b), 0) * ln f: `lng`/`lng2`
    // is the base, the value at the start of the current iteration, and H
    // counts the iteration's visits, so a visit changes H only; the base takes
    // the visits in once per iteration (k_fold).  With ln f = 2^-k the sum is
    // exact and equals the sequential additions of Sec. 2.  REWL_F32 holds
    // ln g itself in `lng1`, rounded at every visit.
    double *lng;      // REWL_FP64 base
    float2 *lng2;     // REWL_F32X2 base (hi, lo)
    float *lng1;      // REWL_F32 ln g
    int32_t *H;       // -1 = never visited
    float *scr;       // exact formats: float screen of the base, base(b) - c_w rounded to
                      //   nearest, c_w a per-walker constant (the walker's ln g at the last
                      //   fold); the decisions screen differences of these values
    DevState *st;
};

// Join scratch (device pointers inside the workspace).
struct JoinScratch {
    double *piece;    // nwin x tstride merged ln g per window
    double *off;      // nwalk: alignment offset of each walker to walker 0 of its window
    double *GE;       // nwin x wE: E marginal of each piece (Eq. 3)
    double *eshift;   // nwin: shift of each piece within its row
    int32_t *efrom, *eto;   // nwin: e range [from, to) each piece covers in its row
    int32_t *ematch;  // nM x max(1, nE-1)
    int32_t *rowok;   // nM
    double *F;        // nM x (N+1): M marginal of each row
    double *mshift;   // nM
    int32_t *mfrom, *mto;   // nM
    int32_t *mmatch;  // max(1, nM-1)
    double *J;        // (N+1) x (N+1) joined table
    double *red;      // reduction scratch (>= 2 * 1024 doubles)
    double *marg;     // N+1 marginal output
    double *gbuf;     // nM x 2 x (N+1) work space of the E matching chains
    double *eslice;   // nwin x wM: rule 1, shift of each M slice of each piece within its row
    double *mslice;   // nM x (N+1): rule 1, shift of each E slice of each row
    double *jk_ref, *jk_sum, *jk_sq;   // jackknife accumulators, (N+1)^2 each
};

// Kernel launchers (rewl_kernels.cu, rewl_join.cu); all return cudaError_t of the launch.
cudaError_t launch_init(const Params &p, const uint8_t *d_init_bytes, cudaStream_t s);
cudaError_t launch_drive(const Params &p, int32_t *d_fail, cudaStream_t s);
cudaError_t launch_sweep(const Params &p, uint64_t ntrials, int walkers_per_block, cudaStream_t s);
// Sweep of walker w alone: one thread of the one-thread-per-walker kernel.
cudaError_t launch_sweep_walker(const Params &p, int w, uint64_t ntrials, cudaStream_t s);
cudaError_t launch_sweep_tree(const Params &p, uint64_t ntrials, int group, int warps, bool smt, cudaStream_t s);
size_t tree_smem_per_warp(const Params &p, bool smt);
cudaError_t launch_exchange(const Params &p, int max_pairs, cudaStream_t s);
cudaError_t launch_flat(const Params &p, cudaStream_t s);
cudaError_t launch_decide(const Params &p, int flags, cudaStream_t s);
// Iteration advance (fold = 1, only when the last check ended an iteration):
// base += H * lnf_done and H -> 0 on visited bins; the screens are refreshed
// in both cases (fold = 0: after the tables were written from the host).
cudaError_t launch_fold(const Params &p, int fold, cudaStream_t s);
cudaError_t launch_digest(const Params &p, unsigned long long *d_out, cudaStream_t s);
cudaError_t launch_rel_diff(const double *a, const double *b, double *out, size_t n, cudaStream_t s);
cudaError_t launch_philox(const uint32_t *d_ctr, uint32_t k0, uint32_t k1, uint32_t *d_out,
                          uint64_t n, cudaStream_t s);
cudaError_t launch_join(const Params &p, const JoinScratch &j, cudaStream_t s);
cudaError_t launch_marginal_e(const Params &p, const JoinScratch &j, cudaStream_t s);
cudaError_t launch_jk_accum(const JoinScratch &j, const double *x, size_t n, int k, cudaStream_t s);
cudaError_t launch_jk_final(const JoinScratch &j, double *mean, double *err, size_t n, int W, cudaStream_t s);

enum : int { DECIDE_XSTEP = 1, DECIDE_CYCLE = 2, DECIDE_CHECK = 4 };

// Host-side geometry and configuration helpers (rewl_api.cu).
struct Dims {
    int precision;
    int L, N, wpr, nwords, nE, nM, W, nwin, nwalk, wE, wM, T;
    long long tstride;
};
void axis_windows(int bins, int n, double overlap, std::vector<int> &lo, std::vector<int> &hi);
bool is_pow2(double x);
bool bin_can_hold(int L, int e, int m);
int check_config(const rewl_config *c, const char **why);
Dims dims_of(const rewl_config *c);

}  // namespace rewl
