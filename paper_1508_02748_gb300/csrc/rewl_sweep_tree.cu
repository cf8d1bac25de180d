// Group-per-walker Wang-Landau sampling with tree speculation (sm_103a).
//
// The trials of one walker form a sequential Markov chain (Eq. 1 and the
// update rule of Sec. 2 of arXiv:1508.02748): each trial depends on the
// accept/reject outcome of the one before.  A group of G lanes (G = 8, 16 or
// 32; 32/G walkers per warp) runs one walker and resolves DEPTH+1 trials per
// step (DEPTH = log2(G) - 1): lanes 0..G-2 form a binary tree; lane l sits at
// depth d = floor(log2(l+1)) and evaluates trial t+d under the history
// h = l + 1 - 2^d (bit k of h = outcome assumed for trial t+k).
//
// Per step every lane
//   1. reads its own trial's site from the ring and the five spins around it
//      from the committed lattice, corrected for the sites its history flips;
//      this gives the move (de, dm) of its trial under its history;
//   2. takes the moves of the earlier trials of its history by shuffle from
//      the lanes that evaluated them (lane 2^k - 1 + (h mod 2^k) for trial k),
//      and walks them to find its current bin and the bins visited;
//   3. decides its own trial (Eq. 1) with the exact ln g values the sequential
//      chain would see there: value(bin) = table(bin) + visits * ln f.
// One ballot then follows the true path from the root; the leaf lane of that
// path commits the DEPTH+1 trials (spin flips, the ln g / H updates of every
// bin visited, the new current bin) and the group adopts its state.
//
// The outcome is the sequential chain itself, trial for trial:
//   - random numbers are drawn per trial index from the TRIAL stream of
//     Philox4x32-10, independent of the state (a ring of 128 trials per
//     walker, refilled 64 at a time from the even trial at or below the
//     launch's first trial);
//   - table(bin) + visits * ln f is evaluated as fma(visits, ln f, table),
//     the same number as the sequential additions whenever ln f = 2^-k (every
//     partial sum is then exact);
//   - decisions are screened in float with a margin that bounds the float
//     rounding, and re-taken in double on near-ties, as in the one-thread
//     sampler.
// The walker's current bin stays in registers (its table value at entry,
// the visits since then) and is written back when the walker leaves it.
#include "rewl_internal.cuh"

namespace rewl {

namespace {

constexpr int RING = 128;   // trials buffered per walker

__device__ __forceinline__ float trunc_f(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const int ex = (int)((hi >> 20) & 0x7FFu);
    if (ex < 897) return 0.0f;
    if (ex > 1150) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u);
    return __uint_as_float((hi & 0x80000000u) | ((uint32_t)(ex - 896) << 23) | ((uint32_t)(b >> 29) & 0x7FFFFFu));
}

__device__ __forceinline__ double unit_open_d(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

struct RingEntry {
    uint32_t ij;   // row << 16 | column of the site
    uint32_t xu;   // acceptance word
    float lnu;     // ln u in float
};

template <int G>
struct TreeShape {
    static constexpr int DEPTH = G == 32 ? 4 : G == 16 ? 3 : G == 8 ? 2 : 1;
};

}  // namespace

template <int WPR, bool SMT, int G>
__global__ void __launch_bounds__(256) k_sweep_tree(Params p, unsigned long long ntrials, int smem_per_walker)
{
    constexpr int DEPTH = TreeShape<G>::DEPTH;
    constexpr int GPW = 32 / G;   // walkers per warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gl = lane & (G - 1), grp = lane / G;
    const unsigned gmask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << (grp * G));
    const int slot = wid * GPW + grp;   // walker slot within the block
    const int w = blockIdx.x * ((blockDim.x >> 5) * GPW) + slot;
    if (w >= p.nwalk) return;
    if (!p.active[w / p.W] || p.st->done) return;

    unsigned char *base = smem_raw + (size_t)slot * smem_per_walker;
    RingEntry *ring = reinterpret_cast<RingEntry *>(base);
    uint32_t *lat = reinterpret_cast<uint32_t *>(base + RING * sizeof(RingEntry));
    const int L = p.L, nwords = L * WPR;
    const int T = p.T;
    double *gl_tab = p.lng + (size_t)w * p.tstride;
    int32_t *gH = p.H + (size_t)w * p.tstride;
    double *tl;
    int32_t *tH;
    if (SMT) {
        tl = reinterpret_cast<double *>(base + RING * sizeof(RingEntry) + ((nwords * 4 + 15) & ~15));
        tH = reinterpret_cast<int32_t *>(tl + T);
        for (int k = gl; k < T; k += G) { tl[k] = gl_tab[k]; tH[k] = gH[k]; }
    } else {
        tl = gl_tab;
        tH = gH;
    }
    for (int k = gl; k < nwords; k += G) lat[k] = p.spins[(size_t)k * p.nwalk + w];
    __syncwarp(gmask);

    const int4 R = p.rect[w / p.W];
    const int wM = p.wM;
    const double lnf = p.st->lnf;
    const float lnf32 = trunc_f(lnf);
    const uint32_t N = (uint32_t)p.N;
    const uint32_t divL = p.divL;

    // this lane's node of the tree
    const int dl = 31 - __clz(gl + 1);
    const int hist = gl + 1 - (1 << dl);

    // committed state (uniform over the group)
    int e = p.we[w], m = p.wm[w];
    int ci = (e - R.x) * wM + (m - R.z);
    double lbase = tl[ci];      // table value of the current bin when entered
    int lq = 0;                 // ln f steps since lbase
    int hq = 0;                 // visits of the current bin not yet in H
    int hbase = tH[ci];
    float base32 = trunc_f(lbase);
    unsigned long long t = p.wt[w];
    const unsigned long long tend = t + ntrials;
    unsigned long long tfill = t & ~1ull;
    int err = 0;

    auto bit = [&](int r, int c) -> uint32_t {
        const int q = (WPR == 1) ? 0 : (c >> 5);
        return (lat[r * WPR + q] >> (c & 31)) & 1u;
    };

    while (t < tend) {
        // ---- refill the ring: 32 Philox calls = 64 trials
        if (tfill < t + 32) {
            #pragma unroll
            for (int r = 0; r < 32 / G; ++r) {
                const unsigned long long c = (tfill >> 1) + (unsigned long long)(gl + r * G);
                const u32x4 x = philox10((uint32_t)c, (uint32_t)(c >> 32), (uint32_t)w, TAG_TRIAL, p.key0, p.key1);
                #pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const uint32_t xs = hh ? x.z : x.x, xu = hh ? x.w : x.y;
                    const uint32_t site = __umulhi(xs, N);
                    const uint32_t i = __umulhi(site, divL);
                    const uint32_t jj = site - i * (uint32_t)L;
                    RingEntry en;
                    en.ij = (i << 16) | jj;
                    en.xu = xu;
                    en.lnu = logf(__fmaf_rn(__uint2float_rn(xu), 0x1p-32f, 0x1p-33f));
                    ring[(2 * c + hh) & (RING - 1)] = en;
                }
            }
            tfill += 64;
            __syncwarp(gmask);
        }
        if (lq >= (1 << 22)) {       // keep the float screen's counts exact
            lbase = fma((double)lq, lnf, lbase);
            lq = 0;
            base32 = trunc_f(lbase);
        }
        const unsigned long long left = tend - t;
        const int D = left > (unsigned long long)DEPTH ? DEPTH : (int)left - 1;

        // ---- 1. own trial under own history
        const RingEntry me = ring[(t + dl) & (RING - 1)];
        int sk[DEPTH];               // sites of the earlier trials
        #pragma unroll
        for (int k = 0; k < DEPTH; ++k) sk[k] = (int)ring[(t + k) & (RING - 1)].ij;
        const int si = (int)(me.ij >> 16), sj = (int)(me.ij & 0xFFFFu);
        const int iu = si == 0 ? L - 1 : si - 1, id = si == L - 1 ? 0 : si + 1;
        const int jl = sj == 0 ? L - 1 : sj - 1, jr = sj == L - 1 ? 0 : sj + 1;
        uint32_t s = bit(si, sj), bu = bit(iu, sj), bd = bit(id, sj), bl = bit(si, jl), br = bit(si, jr);
        #pragma unroll
        for (int k = 0; k < DEPTH; ++k) {
            if (k < dl && ((hist >> k) & 1)) {
                const int fi = sk[k] >> 16, fj = sk[k] & 0xFFFF;
                s ^= (fi == si && fj == sj);
                bu ^= (fi == iu && fj == sj);
                bd ^= (fi == id && fj == sj);
                bl ^= (fi == si && fj == jl);
                br ^= (fi == si && fj == jr);
            }
        }
        const int nup = (int)(bu + bd + bl + br);
        const int de_own = s ? nup - 2 : 2 - nup;
        const int dm_own = s ? -1 : 1;
        const int pack = (de_own + 2) | ((dm_own + 1) << 3);

        // ---- 2. earlier trials of the history: moves from their lanes
        int ce = e, cm = m;
        bool ok = dl <= D;
        int vb[DEPTH];               // bin after each earlier trial
        #pragma unroll
        for (int k = 0; k < DEPTH; ++k) {
            const int src = (1 << k) - 1 + (hist & ((1 << k) - 1));
            const int pk = __shfl_sync(gmask, pack, src, G);
            vb[k] = -1;
            if (k < dl) {
                if ((hist >> k) & 1) {
                    const int en_ = ce + (pk & 7) - 2, mn_ = cm + ((pk >> 3) & 3) - 1;
                    if (en_ < R.x || en_ > R.y || mn_ < R.z || mn_ > R.w) ok = false;  // never accepted
                    ce = en_;
                    cm = mn_;
                }
                vb[k] = (ce - R.x) * wM + (cm - R.z);
            }
        }

        // ---- 3. decision of the own trial (Eq. 1)
        const int en_o = ce + de_own, mn_o = cm + dm_own;
        int acc = 0;
        if (ok && en_o >= R.x && en_o <= R.y && mn_o >= R.z && mn_o <= R.w) {
            const int cb = (ce - R.x) * wM + (cm - R.z);
            const int nbn = (en_o - R.x) * wM + (mn_o - R.z);
            int vcur = 0, vnew = 0;
            #pragma unroll
            for (int k = 0; k < DEPTH; ++k) {
                vcur += (vb[k] == cb);
                vnew += (vb[k] == nbn);
            }
            const bool c0 = cb == ci, n0 = nbn == ci;
            const double cbase = c0 ? lbase : tl[cb];
            const double nbase = n0 ? lbase : tl[nbn];
            const int ccnt = vcur + (c0 ? lq : 0), ncnt = vnew + (n0 ? lq : 0);
            const float cb32 = c0 ? base32 : trunc_f(cbase);
            const float nb32 = n0 ? base32 : trunc_f(nbase);
            const float c32 = __fmaf_rn((float)ccnt, lnf32, cb32);
            const float n32 = __fmaf_rn((float)ncnt, lnf32, nb32);
            const float d32 = c32 - n32;
            const float M = (fabsf(c32) + fabsf(n32) + fabsf(cb32) + fabsf(nb32) + fabsf(me.lnu)) * 0x1p-20f
                          + 0x1p-20f;
            if (me.lnu < d32 - M) {
                acc = 1;
            } else if (me.lnu > d32 + M) {
                acc = 0;
            } else {
                const double delta = fma((double)ccnt, lnf, cbase) - fma((double)ncnt, lnf, nbase);
                acc = (delta >= 0.0 || log(unit_open_d(me.xu)) < delta) ? 1 : 0;
            }
        }

        // ---- follow the true path
        const unsigned bal = (__ballot_sync(gmask, acc) >> (grp * G)) & (G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u));
        int path = 0;
        #pragma unroll
        for (int k = 0; k <= DEPTH; ++k) {
            if (k <= D) {
                const int ln = (1 << k) - 1 + path;
                path |= (int)((bal >> ln) & 1u) << k;
            }
        }
        const int leaf = (1 << D) - 1 + (path & ((1 << D) - 1));

        // ---- commit (leaf lane), then the group adopts the new state
        int n_e = e, n_m = m, n_ci = ci, n_lq = lq, n_hq = hq, n_hb = hbase;
        double n_lb = lbase;
        if (gl == leaf) {
            int fl[DEPTH + 1];
            int vv[DEPTH + 1];
            #pragma unroll
            for (int k = 0; k < DEPTH; ++k) {
                fl[k] = (k < D && ((path >> k) & 1)) ? sk[k] : -1;
                vv[k] = k < D ? vb[k] : -1;
            }
            const bool a = (path >> D) & 1;
            fl[DEPTH] = a ? (int)me.ij : -1;
            const int fe = a ? en_o : ce, fm = a ? mn_o : cm;
            const int C = (fe - R.x) * wM + (fm - R.z);
            vv[DEPTH] = C;     // the visit of the last trial (slot DEPTH stands for trial D)
            #pragma unroll
            for (int k = 0; k <= DEPTH; ++k) {
                if (fl[k] >= 0) {
                    const int fi = fl[k] >> 16, fj = fl[k] & 0xFFFF;
                    atomicXor(&lat[fi * WPR + ((WPR == 1) ? 0 : (fj >> 5))], 1u << (fj & 31));
                }
            }
            // write back every bin visited in this step other than the final one
            int cC = 0;
            bool b0_seen = false;
            #pragma unroll
            for (int k = 0; k <= DEPTH; ++k) {
                const int X = vv[k];
                if (X < 0) continue;
                cC += (X == C);
                b0_seen |= (X == ci);
                bool first = true;
                int cnt = 0;
                #pragma unroll
                for (int k2 = 0; k2 <= DEPTH; ++k2) {
                    if (k2 < k && vv[k2] == X) first = false;
                    cnt += (vv[k2] == X);
                }
                if (first && X != C) {
                    if (X == ci) {
                        const long long hv = (long long)(hbase < 0 ? 0 : hbase) + hq + cnt;
                        if (hv > 0x7FFFFFFFll) err = 1;
                        tl[X] = fma((double)(lq + cnt), lnf, lbase);
                        tH[X] = (int32_t)hv;
                    } else {
                        const int32_t h0 = tH[X];
                        const long long hv = (long long)(h0 < 0 ? 0 : h0) + cnt;
                        if (hv > 0x7FFFFFFFll) err = 1;
                        tl[X] = fma((double)cnt, lnf, tl[X]);
                        tH[X] = (int32_t)hv;
                    }
                }
            }
            if (C == ci) {
                n_lq = lq + cC;
                n_hq = hq + cC;
            } else {
                if (!b0_seen && hq > 0) {      // left the entry bin on the first trial
                    const long long hv = (long long)(hbase < 0 ? 0 : hbase) + hq;
                    if (hv > 0x7FFFFFFFll) err = 1;
                    tl[ci] = fma((double)lq, lnf, lbase);
                    tH[ci] = (int32_t)hv;
                }
                n_ci = C;
                n_lb = tl[C];
                n_hb = tH[C];
                n_lq = cC;
                n_hq = cC;
            }
            n_e = fe;
            n_m = fm;
        }
        __syncwarp(gmask);
        e = __shfl_sync(gmask, n_e, leaf, G);
        m = __shfl_sync(gmask, n_m, leaf, G);
        const int new_ci = __shfl_sync(gmask, n_ci, leaf, G);
        lq = __shfl_sync(gmask, n_lq, leaf, G);
        hq = __shfl_sync(gmask, n_hq, leaf, G);
        hbase = __shfl_sync(gmask, n_hb, leaf, G);
        lbase = __shfl_sync(gmask, n_lb, leaf, G);
        if (new_ci != ci) base32 = trunc_f(lbase);
        ci = new_ci;
        t += (unsigned long long)(D + 1);
    }

    // ---- flush the current bin and the state
    if (gl == 0 && hq > 0) {
        const long long hv = (long long)(hbase < 0 ? 0 : hbase) + hq;
        if (hv > 0x7FFFFFFFll) err = 1;
        tl[ci] = fma((double)lq, lnf, lbase);
        tH[ci] = (int32_t)hv;
    }
    __syncwarp(gmask);
    if (SMT)
        for (int k = gl; k < T; k += G) { gl_tab[k] = tl[k]; gH[k] = tH[k]; }
    for (int k = gl; k < nwords; k += G) p.spins[(size_t)k * p.nwalk + w] = lat[k];
    if (gl == 0) {
        p.we[w] = e;
        p.wm[w] = m;
        p.wt[w] = t;
    }
    err = __any_sync(gmask, err);
    if (gl == 0 && err) atomicOr(&p.st->error, ERR_OVERFLOW);
}

// Shared memory per walker: ring, lattice (16-byte padded) and, when staged,
// the tables.
size_t tree_smem_per_warp(const Params &p, bool smt)
{
    size_t b = RING * sizeof(RingEntry) + (((size_t)p.nwords * 4 + 15) & ~(size_t)15);
    if (smt) b += (size_t)p.T * (sizeof(double) + sizeof(int32_t));
    return (b + 15) & ~(size_t)15;
}

// group: lanes per walker (8, 16 or 32); warps: warps per block.
cudaError_t launch_sweep_tree(const Params &p, uint64_t ntrials, int group, int warps, bool smt, cudaStream_t s)
{
    if (group != 8 && group != 16 && group != 32) group = 32;
    const size_t per = tree_smem_per_warp(p, smt);
    const int gpw = 32 / group;
    if (warps <= 0) warps = smt ? 1 : 4;
    const size_t smem = per * (size_t)gpw * warps;
    const int walkers_per_block = gpw * warps;
    const int blocks = (p.nwalk + walkers_per_block - 1) / walkers_per_block;
    const int threads = 32 * warps;
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, threads, smem, s>>>(p, (unsigned long long)ntrials, (int)per);
        return cudaGetLastError();
    };
#define REWL_TREE_CASES(W_, S_)                                           \
    if (group == 32) return go(k_sweep_tree<W_, S_, 32>);                 \
    if (group == 16) return go(k_sweep_tree<W_, S_, 16>);                 \
    return go(k_sweep_tree<W_, S_, 8>);
    if (p.wpr == 1) {
        if (smt) { REWL_TREE_CASES(1, true) } else { REWL_TREE_CASES(1, false) }
    } else {
        if (smt) { REWL_TREE_CASES(2, true) } else { REWL_TREE_CASES(2, false) }
    }
#undef REWL_TREE_CASES
}

}  // namespace rewl
