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

// ln g access for the two table precisions.
__device__ __forceinline__ double lng_read(const Params &p, size_t i)
{
    if (p.precision == REWL_FP64) return p.lng[i];
    if (p.precision == REWL_F32) return (double)p.lng1[i];
    const float2 v = p.lng2[i];
    return (double)v.x + (double)v.y;
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
// for runs with many walkers, where the walkers alone fill the GPU).
//
// Trial t: site and u from the TRIAL stream; flipping spin s with n_up up
// neighbours moves the bins by de = s (n_up - 2), dm = -s (s = +-1).  A
// proposal outside the window is rejected.  Otherwise, with
// delta = ln g(cur) - ln g(new), it is accepted iff delta >= 0 or
// ln u < delta (Eq. 1 in logarithms).  Then ln g(cur) += ln f and
// H(cur) += 1 for the bin the walker is in (Sec. 2).
//
// The walker's own bin is kept in registers: its table value when entered
// and the visits since; ln g(cur) = value + visits * ln f is formed exactly
// (fma in double, a compensated float pair for REWL_F32X2) -- the same number
// as the sequential additions whenever ln f = 2^-k -- and written back when
// the walker leaves the bin and at the end (a bin left by the very first
// trial of a launch keeps its entries, H = -1 included).  The bin proposed
// is never the current one (dm != 0), so its table entry is up to date.
//
// The decision is screened in float: c = ln g(cur), b = ln g(new) and ln u
// are each known to within a few float roundings (|error| < 2^-21 of their
// sum of magnitudes), so when ln u lies farther than
//     M = 2^-20 (|c| + |b| + |c_0| + |ln u|) + 2^-20
// from c - b the float comparison gives the exact answer; otherwise delta and
// ln u are evaluated in double.  REWL_F32 (plain float, a precision
// demonstration) compares the rounded float values directly.
//
// REG: the lattice (N <= 64, bit i*L + j) is one 64-bit register; otherwise
// it lives in shared memory, word q of row r of thread t at
// sm[(r * wpr + q) * nb + t], so the lanes of a warp never share a bank.
template <int WPR, int PREC, bool REG>
__global__ void __launch_bounds__(128) k_sweep_thread(Params p, unsigned long long ntrials)
{
    using TB = Tab<PREC>;
    using Elem = typename TB::Elem;
    using Val = typename TB::Val;
    extern __shared__ uint32_t sm_all[];
    const int nb = blockDim.x, tid = threadIdx.x;
    const int w = p.walker0 + blockIdx.x * nb + tid;
    if (w >= p.nwalk) return;
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
    Elem *tl = ((PREC == REWL_FP64) ? reinterpret_cast<Elem *>(p.lng)
              : (PREC == REWL_F32X2) ? reinterpret_cast<Elem *>(p.lng2) : reinterpret_cast<Elem *>(p.lng1))
             + (size_t)w * p.tstride;
    int32_t *tH = p.H + (size_t)w * p.tstride;
    const double lnf = p.st->lnf;
    const float lnf32 = trunc_f(lnf);
    const uint32_t N = (uint32_t)p.N;

    int e = p.we[w], m = p.wm[w];
    int ci = (e - R.x) * wM + (m - R.z);
    Val lbase = TB::load(tl, ci);
    float base32 = TB::approx(lbase);
    int lq = 0;          // ln f steps since lbase
    int hq = 0;          // visits not yet in H
    int hbase = tH[ci];
    unsigned long long t = p.wt[w];
    const unsigned long long tend = t + ntrials;
    int err = 0;

    auto bitof = [&](int r, int c) -> uint32_t {
        if (REG) return (uint32_t)(lat >> (r * L + c)) & 1u;
        const int q = (WPR == 1) ? 0 : (c >> 5);
        return (sm[(r * WPR + q) * nb] >> (c & 31)) & 1u;
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
            const Val tn = TB::load(tl, ni);
            const float nb32 = TB::approx(tn);
            bool acc;
            if constexpr (PREC == REWL_F32) {
                acc = lnu < TB::add(lbase, lq, lnf, lnf32) - tn;
            } else {
                const float c32 = __fmaf_rn((float)lq, lnf32, base32);
                const float d32 = c32 - nb32;
                const float M = (fabsf(c32) + fabsf(nb32) + fabsf(base32) + fabsf(lnu)) * 0x1p-20f + 0x1p-20f;
                if (lnu < d32 - M) {
                    acc = true;
                } else if (lnu > d32 + M) {
                    acc = false;
                } else {
                    const double delta = fma((double)lq, lnf, TB::exact(lbase)) - TB::exact(tn);
                    acc = delta >= 0.0 || log(unit_open_d(xu)) < delta;
                }
            }
            if (acc) {
                if (REG) lat ^= 1ull << (i * L + j);
                else sm[(i * WPR + ((WPR == 1) ? 0 : (j >> 5))) * nb] ^= 1u << (j & 31);
                if (hq) {
                    const long long hv = (long long)(hbase < 0 ? 0 : hbase) + hq;
                    if (hv > 0x7FFFFFFFll) err = 1;
                    tl[ci] = TB::add(lbase, lq, lnf, lnf32);
                    tH[ci] = (int32_t)hv;
                }
                ci = ni; lbase = tn; base32 = nb32; lq = 0; hq = 0; hbase = tH[ni];
                e = en; m = mn;
            }
        }
        ++lq;
        ++hq;
        if (lq == (1 << 22)) {              // keep the float screen's counts exact
            lbase = TB::add(lbase, lq, lnf, lnf32);
            base32 = TB::approx(lbase);
            lq = 0;
        }
        ++t;
        if (!(t & 1ull))
            x = philox10((uint32_t)(t >> 1), (uint32_t)(t >> 33), (uint32_t)w, TAG_TRIAL, p.key0, p.key1);
    }
    if (hq) {
        const long long hv = (long long)(hbase < 0 ? 0 : hbase) + hq;
        if (hv > 0x7FFFFFFFll) err = 1;
        tl[ci] = TB::add(lbase, lq, lnf, lnf32);
        tH[ci] = (int32_t)hv;
    }
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
    if (p.sampler == REWL_SAMPLER_WARP) {
        // staged exact tables fold their visit counts once per launch: fewer
        // than 2^22 trials per launch keep every count exact in float
        const uint64_t chunk = (p.smt && p.precision != REWL_F32) ? (1ull << 22) : (1ull << 30);
        while (ntrials > 0) {
            const uint64_t n = ntrials > chunk ? chunk : ntrials;
            const cudaError_t e = launch_sweep_tree(p, n, p.group, wpb, p.smt != 0, s);
            if (e != cudaSuccess) return e;
            ntrials -= n;
        }
        return cudaSuccess;
    }
    if (wpb <= 0) wpb = 32;
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
        const double giX = lng_read(p, bi + (size_t)(eX - RA.x) * p.wM + (mX - RA.z));
        const double giY = lng_read(p, bi + (size_t)(eY - RA.x) * p.wM + (mY - RA.z));
        const double gjY = lng_read(p, bj + (size_t)(eY - RB.x) * p.wM + (mY - RB.z));
        const double gjX = lng_read(p, bj + (size_t)(eX - RB.x) * p.wM + (mX - RB.z));
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

// H reset after an iteration ends: visited bins back to 0, unvisited stay -1.
__global__ void k_reset(Params p)
{
    if (!p.st->advanced) return;
    const size_t n = (size_t)p.nwalk * p.tstride / 4;
    int4 *H4 = reinterpret_cast<int4 *>(p.H);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        int4 v = H4[i];
        v.x = v.x > 0 ? 0 : v.x; v.y = v.y > 0 ? 0 : v.y;
        v.z = v.z > 0 ? 0 : v.z; v.w = v.w > 0 ? 0 : v.w;
        H4[i] = v;
    }
}

cudaError_t launch_reset(const Params &p, cudaStream_t s)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_reset<<<sms * 4, 256, 0, s>>>(p);
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

// ------------------------------------------------------ table copies ----

__global__ void k_tables_to_double(Params p, double *out)
{
    const size_t n = (size_t)p.nwalk * p.T;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t w = i / p.T, b = i % p.T;
        out[i] = lng_read(p, w * p.tstride + b);
    }
}

cudaError_t launch_tables_to_double(const Params &p, double *d_out, cudaStream_t s)
{
    k_tables_to_double<<<1024, 256, 0, s>>>(p, d_out);
    return cudaGetLastError();
}

__global__ void k_tables_from_double(Params p, const double *in)
{
    const size_t n = (size_t)p.nwalk * p.T;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t w = i / p.T, b = i % p.T;
        const double v = in[i];
        if (p.precision == REWL_FP64) {
            p.lng[w * p.tstride + b] = v;
        } else if (p.precision == REWL_F32) {
            p.lng1[w * p.tstride + b] = (float)v;
        } else {
            const float hi = (float)v;
            p.lng2[w * p.tstride + b] = make_float2(hi, (float)(v - (double)hi));
        }
    }
}

cudaError_t launch_tables_from_double(const Params &p, const double *d_in, cudaStream_t s)
{
    k_tables_from_double<<<1024, 256, 0, s>>>(p, d_in);
    return cudaGetLastError();
}

}  // namespace rewl
