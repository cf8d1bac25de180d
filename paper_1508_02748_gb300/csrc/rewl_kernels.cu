// Sampling-side kernels of librewl: initial spins, drive into the windows,
// Wang-Landau trials (Eq. 1 and the update rule of Sec. 2), replica exchange
// (Eq. 2), flatness check (80% rule, Sec. 3) and the iteration advance
// (f -> sqrt f, Sec. 2), for two-dimensional REWL of the periodic L x L Ising
// model (arXiv:1508.02748).
//
// Random draws: Philox4x32-10 with key = seed and counter
//   INIT  (c, 0, walker, 1)       spins of sites 128c .. 128c+127
//   DRIVE (d_lo, d_hi, walker, 2) drive step d
//   TRIAL (c_lo, c_hi, walker, 3) trials 2c (words x, y) and 2c+1 (words z, w):
//                                 site = floor(word * N / 2^32), u = (word + 1/2) 2^-32
//   PERM  (x, pair, i, 4)         Fisher-Yates draw i of exchange sweep x
//   EXCH  (x, pair, k, 5)         acceptance draw of the k-th pair
// pair = 2 * (lower window) + axis.
#include "rewl_tab.cuh"

namespace rewl {

using namespace tab;

namespace {

__device__ __forceinline__ double unit_open(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

// Spin bit of (row r, column c) of this thread's lattice in shared memory.
// Layout: word q of row r of thread t at sm[(r * wpr + q) * nb + t], so the
// 32 lanes of a warp always hit 32 different banks.
template <int WPR>
__device__ __forceinline__ uint32_t sbit(const uint32_t *sm, int nb, int r, int c)
{
    const int q = (WPR == 1) ? 0 : (c >> 5);
    return (sm[(r * WPR + q) * nb] >> (c & 31)) & 1u;
}

// ln g of table entry i: base + max(H, 0) ln f in the exact formats (exact
// in double for the dyadic schedule), the stored value for REWL_F32.
__device__ __forceinline__ double lng_read(const Params &p, size_t i, double lnf)
{
    if (p.precision == REWL_F32) return (double)p.lng1[i];
    const double b = p.precision == REWL_FP64 ? p.lng[i] : Tab<REWL_F32X2>::exact(p.lng2[i]);
    return fma((double)max(p.H[i], 0), lnf, b);
}

}  // namespace

// --------------------------------------------------------------- init ----

// One thread per walker: build the bit-packed lattice (from the INIT stream
// or from given bytes) and its bins e = (E + 2N)/4, m = (M + N)/2 with
// E = -sum of the 2N bonds (right and down neighbours, periodic).
__global__ void k_init(Params p, const uint8_t *init_bytes)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= p.nwalk) return;
    const int L = p.L, N = p.N;
    for (int k = 0; k < p.nwords; ++k) p.spins[(size_t)k * p.nwalk + w] = 0u;
    u32x4 x = {0, 0, 0, 0};
    for (int site = 0; site < N; ++site) {
        uint32_t up;
        if (init_bytes) {
            up = init_bytes[(size_t)w * N + site] != 0;
        } else {
            if ((site & 127) == 0) x = philox10((uint32_t)(site >> 7), 0u, (uint32_t)w, TAG_INIT, p.key0, p.key1);
            const int q = (site >> 5) & 3;
            const uint32_t word = q == 0 ? x.x : q == 1 ? x.y : q == 2 ? x.z : x.w;
            up = (word >> (site & 31)) & 1u;
        }
        const int i = site / L, j = site % L;
        p.spins[(size_t)(i * p.wpr + (j >> 5)) * p.nwalk + w] |= up << (j & 31);
    }
    auto spin = [&](int i, int j) -> int {
        i = (i + L) % L; j = (j + L) % L;
        const uint32_t wd = p.spins[(size_t)(i * p.wpr + (j >> 5)) * p.nwalk + w];
        return ((wd >> (j & 31)) & 1u) ? 1 : -1;
    };
    int E = 0, M = 0;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            const int s = spin(i, j);
            E -= s * spin(i, j + 1);
            E -= s * spin(i + 1, j);
            M += s;
        }
    p.we[w] = (E + 2 * N) / 4;
    p.wm[w] = (M + N) / 2;
    p.wt[w] = 0ull;
    p.wflat[w] = 0;
}

cudaError_t launch_init(const Params &p, const uint8_t *d_init_bytes, cudaStream_t s)
{
    k_init<<<(p.nwalk + 63) / 64, 64, 0, s>>>(p, d_init_bytes);
    return cudaGetLastError();
}

// -------------------------------------------------------------- drive ----

__device__ __forceinline__ int l1_to_rect(int4 R, int e, int m)
{
    int d = 0;
    d += e < R.x ? R.x - e : 0;
    d += e > R.y ? e - R.y : 0;
    d += m < R.z ? R.z - m : 0;
    d += m > R.w ? m - R.w : 0;
    return d;
}

// One thread per walker: random single flips accepted iff the L1 distance of
// (e, m) to the walker's window does not grow, until inside; a walker still
// outside after drive_budget steps sets *fail.
__global__ void k_drive(Params p, int32_t *fail)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= p.nwalk) return;
    const int win = w / p.W;
    if (!p.active[win]) return;
    const int4 R = p.rect[win];
    const int L = p.L;
    int e = p.we[w], m = p.wm[w];
    auto word_ptr = [&](int i, int j) -> uint32_t * {
        return p.spins + (size_t)(i * p.wpr + (j >> 5)) * p.nwalk + w;
    };
    auto bit = [&](int i, int j) -> uint32_t { return (*word_ptr(i, j) >> (j & 31)) & 1u; };
    uint64_t d = 0;
    int dist = l1_to_rect(R, e, m);
    while (dist > 0) {
        if (d >= p.drive_budget) { atomicExch(fail, 1); return; }
        const u32x4 x = philox10((uint32_t)d, (uint32_t)(d >> 32), (uint32_t)w, TAG_DRIVE, p.key0, p.key1);
        const int site = (int)__umulhi(x.x, (uint32_t)p.N);
        const int i = site / L, j = site - (site / L) * L;
        const uint32_t s = bit(i, j);
        const uint32_t nup = bit(i == 0 ? L - 1 : i - 1, j) + bit(i == L - 1 ? 0 : i + 1, j)
                           + bit(i, j == 0 ? L - 1 : j - 1) + bit(i, j == L - 1 ? 0 : j + 1);
        const int de = s ? (int)nup - 2 : 2 - (int)nup;
        const int dm = s ? -1 : 1;
        const int nd = l1_to_rect(R, e + de, m + dm);
        if (nd <= dist) {
            *word_ptr(i, j) ^= 1u << (j & 31);
            e += de; m += dm; dist = nd;
        }
        ++d;
    }
    p.we[w] = e;
    p.wm[w] = m;
}

cudaError_t launch_drive(const Params &p, int32_t *d_fail, cudaStream_t s)
{
    k_drive<<<(p.nwalk + 63) / 64, 64, 0, s>>>(p, d_fail);
    return cudaGetLastError();
}

// -------------------------------------------------------------- sweep ----

// ntrials Wang-Landau trials per walker, one thread per walker (the sampler
// for runs with many walkers, where the walkers alone fill the GPU, the plain
// one-walker-per-launch form, and plain-float tables).
//
// Trial t: site and u from the TRIAL stream; flipping spin s with n_up up
// neighbours moves the bins by de = s (n_up - 2), dm = -s (s = +-1).  A
// proposal outside the window is rejected.  Otherwise, with
// delta = ln g(cur) - ln g(new), it is accepted iff delta >= 0 or
// ln u < delta (Eq. 1 in logarithms).  Then ln g(cur) += ln f and
// H(cur) += 1 for the bin the walker is in (Sec. 2).
//
// Exact formats: ln g(b) = base(b) + max(H(b), 0) ln f with the base fixed
// during the iteration, so a visit is H + 1 alone.  The walker's own count is
// kept in a register and written back when it leaves the bin and at the end
// (a bin left by the very first trial of a launch keeps its H, -1 included).
// The proposed bin is never the current one (dm != 0), so its H is up to
// date.  The decision is screened in float from the screens S (base minus a
// per-walker constant, rounded): with c = S_c + n_c ln f and b = S_b + n_b
// ln f in float, when ln u lies farther than
//     M = 2^-20 (|c| + |b| + |S_c| + |S_b| + |ln u|) + 2^-20
// from c - b the float comparison gives the exact answer (the error bound is
// that of the tree sampler); otherwise delta and ln u are evaluated in
// double.  REWL_F32 (plain float, a precision demonstration) keeps ln g
// itself, adds ln f with a float rounding at every visit and compares the
// rounded values directly.
//
// REG: the lattice (N <= 64, bit i*L + j) is one 64-bit register; otherwise
// it lives in shared memory, word q of row r of thread t at
// sm[(r * wpr + q) * nb + t], so the lanes of a warp never share a bank.
template <int WPR, int PREC, bool REG>
__global__ void __launch_bounds__(128) k_sweep_thread(Params p, unsigned long long ntrials)
{
    using TB = Tab<PREC>;
    using Elem = typename TB::Elem;
    extern __shared__ uint32_t sm_all[];
    const int nb = blockDim.x, tid = threadIdx.x;
    const int w = p.walker0 + blockIdx.x * nb + tid;
    if (w >= p.nwalk || ntrials == 0) return;
    if (!p.active[w / p.W] || p.st->done) return;
    uint32_t *sm = sm_all + tid;
    const int L = p.L, nwords = L * WPR;
    unsigned long long lat = 0;
    if (REG) {
        for (int r = 0; r < L; ++r) lat |= (unsigned long long)p.spins[(size_t)r * p.nwalk + w] << (r * L);
    } else {
        for (int k = 0; k < nwords; ++k) sm[k * nb] = p.spins[(size_t)k * p.nwalk + w];
    }

    const int4 R = p.rect[w / p.W];
    const int wM = p.wM;
    const unsigned spanE = (unsigned)(R.y - R.x), spanM = (unsigned)(R.w - R.z);
    const Elem *gb = reinterpret_cast<const Elem *>(PREC == REWL_FP64 ? (const void *)p.lng
                                                  : PREC == REWL_F32X2 ? (const void *)p.lng2 : (const void *)p.lng1)
                   + (size_t)w * p.tstride;
    float *t1 = p.lng1 + (size_t)w * p.tstride;      // REWL_F32 values
    const float *S = p.scr + (size_t)w * p.tstride;  // exact formats
    int32_t *tH = p.H + (size_t)w * p.tstride;
    const double lnf = p.st->lnf;
    const float lnf32 = __double2float_rn(lnf);
    const uint32_t N = (uint32_t)p.N;

    int e = p.we[w], m = p.wm[w];
    int ci = (e - R.x) * wM + (m - R.z);
    int lq;              // exact formats: H of the current bin; REWL_F32: visits since v1
    int hq = 0;          // visits not yet written to H
    int hbase = tH[ci];  // REWL_F32: H of the current bin when entered
    float base32;        // exact formats: screen of the current bin
    float v1 = 0.0f;     // REWL_F32: value of the current bin when entered
    if (PREC == REWL_F32) {
        lq = 0;
        v1 = t1[ci];
        base32 = v1;
    } else {
        lq = max(hbase, 0);
        base32 = S[ci];
    }
    unsigned long long t = p.wt[w];
    const unsigned long long tend = t + ntrials;
    int err = 0;

    auto bitof = [&](int r, int c) -> uint32_t {
        if (REG) return (uint32_t)(lat >> (r * L + c)) & 1u;
        const int q = (WPR == 1) ? 0 : (c >> 5);
        return (sm[(r * WPR + q) * nb] >> (c & 31)) & 1u;
    };
    auto flush = [&]() {
        if (PREC == REWL_F32) {
            const long long hv = (long long)(hbase < 0 ? 0 : hbase) + hq;
            if (hv > 0x7FFFFFFFll) err = 1;
            t1[ci] = f32_visits(v1, lq, lnf32);
            tH[ci] = (int32_t)hv;
        } else {
            tH[ci] = lq;
            err |= lq < 0;
        }
    };

    u32x4 x = philox10((uint32_t)(t >> 1), (uint32_t)(t >> 33), (uint32_t)w, TAG_TRIAL, p.key0, p.key1);
    while (t < tend) {
        const bool odd = t & 1ull;
        const uint32_t xs = odd ? x.z : x.x;
        const uint32_t xu = odd ? x.w : x.y;
        const float lnu = logf(__fmaf_rn(__uint2float_rn(xu), 0x1p-32f, 0x1p-33f));
        const uint32_t site = __umulhi(xs, N);
        const int i = (int)__umulhi(site, p.divL);
        const int j = (int)site - i * L;
        const int iu = i == 0 ? L - 1 : i - 1, id = i == L - 1 ? 0 : i + 1;
        const int jl = j == 0 ? L - 1 : j - 1, jr = j == L - 1 ? 0 : j + 1;
        const uint32_t sp = bitof(i, j);
        const int nup = (int)(bitof(iu, j) + bitof(id, j) + bitof(i, jl) + bitof(i, jr));
        const int en = e + (sp ? nup - 2 : 2 - nup);
        const int mn = m + (sp ? -1 : 1);
        if ((unsigned)(en - R.x) <= spanE && (unsigned)(mn - R.z) <= spanM) {
            const int ni = (en - R.x) * wM + (mn - R.z);
            bool acc;
            int hn = 0;
            float vn = 0.0f;
            if constexpr (PREC == REWL_F32) {
                vn = t1[ni];
                acc = lnu < f32_visits(v1, lq, lnf32) - vn;
            } else {
                hn = max(tH[ni], 0);
                vn = S[ni];
                const float c32 = __fmaf_rn(__int2float_rn(lq), lnf32, base32);
                const float n32 = __fmaf_rn(__int2float_rn(hn), lnf32, vn);
                const float d32 = __fsub_rn(c32, n32);
                const float M = __fmaf_rn(fabsf(c32) + fabsf(n32) + fabsf(base32) + fabsf(vn) + fabsf(lnu),
                                          0x1p-20f, 0x1p-20f);
                if (lnu < d32 - M) {
                    acc = true;
                } else if (lnu > d32 + M) {
                    acc = false;
                } else {
                    const double delta = fma((double)lq, lnf, TB::exact(gb[ci])) - fma((double)hn, lnf, TB::exact(gb[ni]));
                    acc = delta >= 0.0 || log(unit_open_d(xu)) < delta;
                }
            }
            if (acc) {
                if (REG) lat ^= 1ull << (i * L + j);
                else sm[(i * WPR + ((WPR == 1) ? 0 : (j >> 5))) * nb] ^= 1u << (j & 31);
                if (hq) flush();
                ci = ni; hq = 0;
                if (PREC == REWL_F32) {
                    v1 = vn; lq = 0; hbase = tH[ni];
                } else {
                    lq = hn; base32 = vn;
                }
                e = en; m = mn;
            }
        }
        ++lq;
        ++hq;
        if (PREC == REWL_F32 && lq == 64) {   // keep the per-visit roundings short
            v1 = f32_visits(v1, lq, lnf32);
            lq = 0;
        }
        ++t;
        if (!(t & 1ull))
            x = philox10((uint32_t)(t >> 1), (uint32_t)(t >> 33), (uint32_t)w, TAG_TRIAL, p.key0, p.key1);
    }
    if (hq) flush();
    p.we[w] = e;
    p.wm[w] = m;
    p.wt[w] = t;
    if (REG) {
        for (int r = 0; r < L; ++r)
            p.spins[(size_t)r * p.nwalk + w] = (uint32_t)(lat >> (r * L)) & (uint32_t)((1ull << L) - 1);
    } else {
        for (int k = 0; k < nwords; ++k) p.spins[(size_t)k * p.nwalk + w] = sm[k * nb];
    }
    if (err) atomicOr(&p.st->error, ERR_OVERFLOW);
}

namespace {

// blocks x wpb threads of k_sweep_thread, walkers p.walker0 onwards.
cudaError_t launch_thread(const Params &p, int blocks, int wpb, uint64_t ntrials, cudaStream_t s)
{
    const bool reg = p.N <= 64 && p.wpr == 1;
    const size_t smem = reg ? 0 : (size_t)p.nwords * wpb * sizeof(uint32_t);
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, wpb, smem, s>>>(p, (unsigned long long)ntrials);
        return cudaGetLastError();
    };
#define REWL_THREAD_P(P_)                                              \
    if (reg) return go(k_sweep_thread<1, P_, true>);                   \
    if (p.wpr == 1) return go(k_sweep_thread<1, P_, false>);           \
    return go(k_sweep_thread<2, P_, false>);
    if (p.precision == REWL_FP64) { REWL_THREAD_P(REWL_FP64) }
    if (p.precision == REWL_F32X2) { REWL_THREAD_P(REWL_F32X2) }
    REWL_THREAD_P(REWL_F32)
#undef REWL_THREAD_P
}

}  // namespace

cudaError_t launch_sweep(const Params &p, uint64_t ntrials, int wpb, cudaStream_t s)
{
    // the tree sampler serves the exact table formats; plain-float tables
    // (a precision demonstration) always run on the thread sampler
    if (p.sampler == REWL_SAMPLER_WARP && p.precision != REWL_F32) {
        const uint64_t chunk = 1ull << 30;
        while (ntrials > 0) {
            const uint64_t n = ntrials > chunk ? chunk : ntrials;
            const cudaError_t e = launch_sweep_tree(p, n, p.group, wpb, p.smt != 0, s);
            if (e != cudaSuccess) return e;
            ntrials -= n;
        }
        return cudaSuccess;
    }
    if (p.sampler == REWL_SAMPLER_WARP || wpb <= 0) wpb = 32;
    return launch_thread(p, (p.nwalk + wpb - 1) / wpb, wpb, ntrials, s);
}

cudaError_t launch_sweep_walker(const Params &p, int w, uint64_t ntrials, cudaStream_t s)
{
    Params q = p;
    q.walker0 = w;
    return launch_thread(q, 1, 1, ntrials, s);
}

// ----------------------------------------------------------- exchange ----

// One block per window pair of the current phase (phase = xstep mod 4:
// E-even, E-odd, M-even, M-odd).  Walker k of the lower window pairs with
// walker pi(k) of the upper one, pi a Fisher-Yates permutation from the PERM
// stream.  A pair is attempted only if each configuration lies in the other
// window; it is accepted with min[1, g_i(X)/g_i(Y) g_j(Y)/g_j(X)] (Eq. 2),
// X, Y the configurations of walkers i (lower) and j (upper) before the swap,
// each g the walker's own table.  On acceptance the lattices and bins swap;
// no g or H is updated.
__global__ void k_exchange(Params p)
{
    extern __shared__ int perm[];
    __shared__ unsigned long long s_att, s_acc;
    if (p.st->done) return;
    const unsigned long long xs = p.st->xstep;
    const int phase = (int)(xs & 3ull), axis = phase >> 1, parity = phase & 1;
    const int nA = axis == 0 ? p.nE : p.nM;
    const int nO = axis == 0 ? p.nM : p.nE;
    const int per = (nA - parity) / 2;
    if (per <= 0 || (int)blockIdx.x >= per * nO) return;
    const int q = blockIdx.x % per, o = blockIdx.x / per;
    const int lo = parity + 2 * q;
    const int a = axis == 0 ? lo : o, b = axis == 0 ? o : lo;
    const int A = b * p.nE + a;
    const int B = axis == 0 ? A + 1 : A + p.nE;
    if (!p.active[A] || !p.active[B]) return;
    const int W = p.W;
    const uint32_t pair = (uint32_t)(2 * A + axis);
    if (threadIdx.x == 0) {
        for (int k = 0; k < W; ++k) perm[k] = k;
        for (int i = W - 1; i >= 1; --i) {
            const u32x4 r = philox10((uint32_t)xs, pair, (uint32_t)i, TAG_PERM, p.key0, p.key1);
            const int j = (int)__umulhi(r.x, (uint32_t)(i + 1));
            const int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
        }
        s_att = 0ull; s_acc = 0ull;
    }
    __syncthreads();
    const int4 RA = p.rect[A], RB = p.rect[B];
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        const int wi = A * W + k, wj = B * W + perm[k];
        const int eX = p.we[wi], mX = p.wm[wi], eY = p.we[wj], mY = p.wm[wj];
        const bool xinB = eX >= RB.x && eX <= RB.y && mX >= RB.z && mX <= RB.w;
        const bool yinA = eY >= RA.x && eY <= RA.y && mY >= RA.z && mY <= RA.w;
        if (!xinB || !yinA) continue;
        const size_t bi = (size_t)wi * p.tstride, bj = (size_t)wj * p.tstride;
        const double lnf = p.st->lnf;
        const double giX = lng_read(p, bi + (size_t)(eX - RA.x) * p.wM + (mX - RA.z), lnf);
        const double giY = lng_read(p, bi + (size_t)(eY - RA.x) * p.wM + (mY - RA.z), lnf);
        const double gjY = lng_read(p, bj + (size_t)(eY - RB.x) * p.wM + (mY - RB.z), lnf);
        const double gjX = lng_read(p, bj + (size_t)(eX - RB.x) * p.wM + (mX - RB.z), lnf);
        const double lnP = (giX - giY) + (gjY - gjX);
        const u32x4 r = philox10((uint32_t)xs, pair, (uint32_t)k, TAG_EXCH, p.key0, p.key1);
        atomicAdd(&s_att, 1ull);
        if (lnP >= 0.0 || log(unit_open(r.x)) < lnP) {
            for (int word = 0; word < p.nwords; ++word) {
                uint32_t *pa = p.spins + (size_t)word * p.nwalk + wi;
                uint32_t *pb = p.spins + (size_t)word * p.nwalk + wj;
                const uint32_t tmp = *pa; *pa = *pb; *pb = tmp;
            }
            p.we[wi] = eY; p.wm[wi] = mY;
            p.we[wj] = eX; p.wm[wj] = mX;
            atomicAdd(&s_acc, 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_att) {
        atomicAdd(&p.st->exch_attempts, s_att);
        atomicAdd(&p.st->exch_accepts, s_acc);
    }
}

cudaError_t launch_exchange(const Params &p, int max_pairs, cudaStream_t s)
{
    if (max_pairs <= 0) return cudaSuccess;
    const int threads = p.W <= 32 ? 32 : (p.W <= 128 ? 128 : 256);
    k_exchange<<<max_pairs, threads, (size_t)p.W * sizeof(int), s>>>(p);
    return cudaGetLastError();
}

// --------------------------------------------------------------- flat ----

// One block per walker: over visited bins (H >= 0), n_seen, sum H and min H;
// flat iff min H * n_seen * 10^6 >= round(flatness * 10^6) * sum H (the 80%
// rule of Sec. 3 in exact integers).
__global__ void __launch_bounds__(256) k_flat(Params p)
{
    if (p.st->done) return;
    const int w = blockIdx.x;
    if (!p.active[w / p.W]) return;
    const int32_t *H = p.H + (size_t)w * p.tstride;
    long long cnt = 0, sum = 0;
    int mn = 0x7FFFFFFF;
    const int T = p.T;
    const int T4 = T & ~3;
    const int4 *H4 = reinterpret_cast<const int4 *>(H);
    for (int i = threadIdx.x; i < T4 / 4; i += blockDim.x) {
        const int4 v = H4[i];
        if (v.x >= 0) { ++cnt; sum += v.x; mn = min(mn, v.x); }
        if (v.y >= 0) { ++cnt; sum += v.y; mn = min(mn, v.y); }
        if (v.z >= 0) { ++cnt; sum += v.z; mn = min(mn, v.z); }
        if (v.w >= 0) { ++cnt; sum += v.w; mn = min(mn, v.w); }
    }
    for (int i = T4 + threadIdx.x; i < T; i += blockDim.x) {
        const int v = H[i];
        if (v >= 0) { ++cnt; sum += v; mn = min(mn, v); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
    }
    __shared__ long long s_cnt[8], s_sum[8];
    __shared__ int s_mn[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { s_cnt[wid] = cnt; s_sum[wid] = sum; s_mn[wid] = mn; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 1; k < nw; ++k) { cnt += s_cnt[k]; sum += s_sum[k]; mn = min(mn, s_mn[k]); }
        const int flat = cnt > 0 && (long long)mn * cnt * 1000000ll >= p.flat_q * sum;
        p.wflat[w] = flat;
        if (flat) atomicAdd(&p.st->nflat, 1);
    }
}

cudaError_t launch_flat(const Params &p, cudaStream_t s)
{
    k_flat<<<p.nwalk, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------- decide ----

// Single thread: advances the exchange/cycle counters and, on a check,
// ends the iteration when every walker of a non-empty window is flat:
// ln f <- ln f * factor, or done once the finished iteration had
// ln f <= lnf_final (Sec. 2: all walkers move on together; stop at f_final).
__global__ void k_decide(Params p, int flags)
{
    DevState *st = p.st;
    if (st->done) { st->advanced = 0; return; }
    if (flags & DECIDE_XSTEP) st->xstep += 1ull;
    if (flags & DECIDE_CYCLE) st->cycle += 1ull;
    st->advanced = 0;
    if (flags & DECIDE_CHECK) {
        const int nf = st->nflat;
        st->nflat_last = nf;
        st->nflat = 0;
        if (nf == p.n_active_walkers) {
            st->advanced = 1;
            st->iter += 1;
            st->lnf_done = st->lnf;
            if (st->lnf <= p.lnf_final) st->done = 1;
            else st->lnf = st->lnf * p.lnf_factor;
        }
    }
}

cudaError_t launch_decide(const Params &p, int flags, cudaStream_t s)
{
    k_decide<<<1, 1, 0, s>>>(p, flags);
    return cudaGetLastError();
}

// Iteration advance (f -> sqrt f, Sec. 2), one block per walker.  Exact
// formats: the finished iteration's visits enter the base, base += H ln f
// (ln f of that iteration; exact for the dyadic schedule), and H goes back to
// 0 on visited bins (-1, never visited, stays).  The screens are refreshed:
// S = base - c_w rounded to float, c_w = ln g of the walker's current bin.
// REWL_F32: H reset only.  fold = 0 refreshes the screens alone (after the
// tables were written from the host); fold = 1 does nothing unless the last
// check ended an iteration.
template <int PREC>
__global__ void __launch_bounds__(256) k_fold(Params p, int fold)
{
    using TB = Tab<PREC>;
    using Elem = typename TB::Elem;
    if (fold && !p.st->advanced) return;
    const int w = blockIdx.x;
    int32_t *H = p.H + (size_t)w * p.tstride;
    const int T = p.T;
    if (PREC == REWL_F32) {
        if (fold)
            for (int k = threadIdx.x; k < T; k += blockDim.x) H[k] = H[k] > 0 ? 0 : H[k];
        return;
    }
    Elem *B = reinterpret_cast<Elem *>(PREC == REWL_FP64 ? (void *)p.lng : (void *)p.lng2) + (size_t)w * p.tstride;
    float *S = p.scr + (size_t)w * p.tstride;
    const double lnf = fold ? p.st->lnf_done : p.st->lnf;
    __shared__ double s_c;
    if (threadIdx.x == 0) {
        const int4 R = p.rect[w / p.W];
        const int e = p.we[w], m = p.wm[w];
        double c = 0.0;
        if (p.active[w / p.W] && e >= R.x && e <= R.y && m >= R.z && m <= R.w) {
            const int ci = (e - R.x) * p.wM + (m - R.z);
            c = fma((double)max(H[ci], 0), lnf, TB::exact(B[ci]));
        }
        s_c = c;
    }
    __syncthreads();
    const double c = s_c;
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        double v = TB::exact(B[k]);
        if (fold) {
            const int h = H[k];
            if (h > 0) {
                v = fma((double)h, lnf, v);
                B[k] = TB::from(v);
                H[k] = 0;
            }
        }
        S[k] = __double2float_rn(v - c);
    }
}

cudaError_t launch_fold(const Params &p, int fold, cudaStream_t s)
{
    if (p.nwalk <= 0) return cudaSuccess;
    if (p.precision == REWL_FP64) k_fold<REWL_FP64><<<p.nwalk, 256, 0, s>>>(p, fold);
    else if (p.precision == REWL_F32X2) k_fold<REWL_F32X2><<<p.nwalk, 256, 0, s>>>(p, fold);
    else k_fold<REWL_F32><<<p.nwalk, 256, 0, s>>>(p, fold);
    return cudaGetLastError();
}

// Order-independent digest of every walker's tables: for each entry, the bit
// pattern of its ln g as a double (base + max(H, 0) ln f in the exact
// formats) and its H are mixed with the entry's index by a 64-bit finaliser
// (the multiply-xorshift steps of splitmix64) and summed modulo 2^64, so two
// runs have equal digests when their tables hold the same values.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_digest(Params p, unsigned long long *out)
{
    const size_t n = (size_t)p.nwalk * p.T;
    const double lnf = p.st->lnf;
    unsigned long long acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t w = i / p.T, b = i % p.T;
        const size_t q = w * p.tstride + b;
        const double v = lng_read(p, q, lnf);
        const unsigned long long h = (unsigned long long)(uint32_t)p.H[q];
        acc += mix64((unsigned long long)__double_as_longlong(v) ^ mix64(i)) + mix64(h + 0x9E3779B97F4A7C15ull * i);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

cudaError_t launch_digest(const Params &p, unsigned long long *d_out, cudaStream_t s)
{
    k_digest<<<1024, 256, 0, s>>>(p, d_out);
    return cudaGetLastError();
}

// ------------------------------------------------------------- philox ----

__global__ void k_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, uint64_t n)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const u32x4 r = philox10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
        out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
    }
}

cudaError_t launch_philox(const uint32_t *d_ctr, uint32_t k0, uint32_t k1, uint32_t *d_out, uint64_t n,
                          cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_philox<<<(unsigned)blocks, 256, 0, s>>>(d_ctr, k0, k1, d_out, n);
    return cudaGetLastError();
}

}  // namespace rewl
