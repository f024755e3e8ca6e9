// Tree on the real parts of the points, level restriction, complexified
// centres and Lists 1-4 (Sec. 6.1-6.2), built on the GPU.
//
// Representation: the tree is the Morton-ordered list of its leaves
// (level, prefix, [start, end) into the sorted points). Splitting a leaf
// replaces it by its non-empty children in place (count + scan + emit), so
// refinement, level restriction and the forced split down to the top
// expansion level are all "split these leaves" passes. Boxes of every level
// are then the distinct level-l prefixes of the leaves at level >= l.
//
// Conventions shared with the specification of the method:
//   root square: centre (min+max)/2, width W = max extent * (1 + 2^-20);
//   q = floor((x - lo)/W * 2^B) clamped, B = 31 (2D) / 21 (3D), computed
//   with explicitly rounded operations (no contraction);
//   Morton key: bits of q interleaved, x lowest; stable LSD radix sort;
//   near(a, b): ||x_a - x_b||_inf <= k/2 (w_a + w_b) in integer arithmetic;
//   level restriction: no leaf near a box two levels finer;
//   Lists as in Sec. 6.2 with the top expansion level l0.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "cfmm_common.cuh"
#include "kernels.cuh"

namespace cfmm {

// Optional host-side phase timing of plan construction (CFMM_PLAN_PROFILE=1):
// each phase is synchronised and its wall time printed to stderr.

// ---------------------------------------------------------------------------
// exclusive scan of int32 (any length), returns the total
// ---------------------------------------------------------------------------
static constexpr int kScanThreads = 512;
static constexpr int kScanItems = 4;
static constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_tile(const int* __restrict__ in, int* __restrict__ out, int n,
                            int* __restrict__ block_sums) {
    __shared__ int warp_tot[kScanThreads / 32];
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = xi - x;
        if (lane == kScanThreads / 32 - 1 && block_sums) block_sums[blockIdx.x] = xi;
    }
    __syncthreads();
    int run = warp_tot[w] + incl - s;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ block_off) {
    int idx = blockIdx.x * kScanTile + threadIdx.x;
    int add = block_off[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i, idx += kScanThreads)
        if (idx < n) out[idx] += add;
}

// exclusive scan in -> out (must not alias), asynchronous
static void scan_exclusive_async(const int* in, int* out, int n, cudaStream_t st) {
    if (n <= 0) return;
    int nb = (n + kScanTile - 1) / kScanTile;
    int* sums = plan_scratch().take_n<int>(nb);
    k_scan_tile<<<nb, kScanThreads, 0, st>>>(in, out, n, sums);
    CFMM_LAUNCHED();
    if (nb > 1) {
        int* sums_x = plan_scratch().take_n<int>(nb);
        scan_exclusive_async(sums, sums_x, nb, st);
        k_scan_add<<<nb, kScanThreads, 0, st>>>(out, n, sums_x);
        CFMM_LAUNCHED();
    }
}

// exclusive scan; returns the total (synchronises the stream)
static int64_t scan_exclusive(const int* in, int* out, int n, cudaStream_t st) {
    if (n <= 0) return 0;
    scan_exclusive_async(in, out, n, st);
    // total = last exclusive value + last input
    int last_out = 0, last_in = 0;
    CFMM_CUDA(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    return (int64_t)last_out + last_in;
}

// ---------------------------------------------------------------------------
// LSD radix sort of (uint64 key, int32 value), 4-bit digits, stable
// ---------------------------------------------------------------------------
static constexpr int kSortThreads = 256;
static constexpr int kSortItems = 8;                 // chunks per tile
static constexpr int kSortTile = kSortThreads * kSortItems;

static constexpr int kRadixBits = 8;                // digit width of one pass
static constexpr int kRadix = 1 << kRadixBits;

__global__ void k_sort_hist(const uint64_t* __restrict__ keys, int n, int shift,
                            int* __restrict__ hist, int ntiles) {
    __shared__ int h[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) h[d] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    for (int c = 0; c < kSortItems; ++c) {
        int i = base + c * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[d * ntiles + blockIdx.x] = h[d];
}

// stable scatter of one digit: within a tile, items keep their order (chunk
// by chunk, warp by warp, and by lane rank among equal digits in a warp)
__global__ void k_sort_scatter(const uint64_t* __restrict__ kin, const int* __restrict__ vin,
                               uint64_t* __restrict__ kout, int* __restrict__ vout, int n,
                               int shift, const int* __restrict__ offs, int ntiles) {
    __shared__ int run[kRadix];
    __shared__ int wcnt[kSortThreads / 32][kRadix];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) run[d] = offs[d * ntiles + blockIdx.x];
    int base = blockIdx.x * kSortTile;
    __syncthreads();
    for (int c = 0; c < kSortItems; ++c) {
        int i = base + c * kSortThreads + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int val = valid ? vin[i] : 0;
        unsigned dig = valid ? (unsigned)((key >> shift) & (kRadix - 1)) : (unsigned)kRadix;
        unsigned same = __match_any_sync(0xffffffffu, dig);
        unsigned lt = (1u << lane) - 1u;
        int rank = __popc(same & lt);
        for (int d = lane; d < kRadix; d += 32) wcnt[w][d] = 0;
        __syncwarp();
        if (valid && rank == 0) wcnt[w][dig] = __popc(same);
        __syncthreads();
        if (valid) {
            int pre = run[dig];
            for (int ww = 0; ww < w; ++ww) pre += wcnt[ww][dig];
            int pos = pre + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
            int s2 = 0;
            for (int ww = 0; ww < kSortThreads / 32; ++ww) s2 += wcnt[ww][d];
            run[d] += s2;
        }
        __syncthreads();
    }
}

// sorts keys (in place, via ping-pong) with payload; nbits = significant bits
static void radix_sort(DevBuf<uint64_t>& keys, DevBuf<int>& vals, int n, int nbits, cudaStream_t st) {
    if (n <= 1) return;
    Scratch& scr = plan_scratch();
    int ntiles = (n + kSortTile - 1) / kSortTile;
    uint64_t* k2 = scr.take_n<uint64_t>(n);
    int* v2 = scr.take_n<int>(n);
    int* hist = scr.take_n<int>((size_t)kRadix * ntiles);
    int* offs = scr.take_n<int>((size_t)kRadix * ntiles);
    uint64_t *ka = keys.get(), *kb = k2;
    int *va = vals.get(), *vb = v2;
    int passes = (nbits + kRadixBits - 1) / kRadixBits;
    for (int p = 0; p < passes; ++p) {
        int shift = kRadixBits * p;
        k_sort_hist<<<ntiles, kSortThreads, 0, st>>>(ka, n, shift, hist, ntiles);
        CFMM_LAUNCHED();
        scan_exclusive_async(hist, offs, kRadix * ntiles, st);
        k_sort_scatter<<<ntiles, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, offs, ntiles);
        CFMM_LAUNCHED();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys.get()) {
        CFMM_CUDA(cudaMemcpyAsync(keys.get(), ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
        CFMM_CUDA(cudaMemcpyAsync(vals.get(), va, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
    }
    CFMM_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// bounding box, keys, gather
// ---------------------------------------------------------------------------
__global__ void k_bbox(const double* __restrict__ re, int64_t n, int dim, double* __restrict__ part) {
    // part[blockIdx][2*dim]: min then max per axis
    __shared__ double smn[256][3], smx[256][3];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < dim; ++d) {
            double v = re[i * dim + d];
            mn[d] = fmin(mn[d], v);
            mx[d] = fmax(mx[d], v);
        }
    }
    for (int d = 0; d < 3; ++d) {
        smn[threadIdx.x][d] = mn[d];
        smx[threadIdx.x][d] = mx[d];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int d = 0; d < 3; ++d) {
                smn[threadIdx.x][d] = fmin(smn[threadIdx.x][d], smn[threadIdx.x + s][d]);
                smx[threadIdx.x][d] = fmax(smx[threadIdx.x][d], smx[threadIdx.x + s][d]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < dim; ++d) {
            part[blockIdx.x * 2 * dim + d] = smn[0][d];
            part[blockIdx.x * 2 * dim + dim + d] = smx[0][d];
        }
}

__global__ void k_nonfinite(const double* __restrict__ a, int64_t m, int* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) atomicOr(flag, 1);
}

__device__ __forceinline__ uint64_t spread_bits(uint64_t q, int dim, int B) {
    uint64_t k = 0;
    for (int b = 0; b < B; ++b) k |= ((q >> b) & 1ull) << (b * dim);
    return k;
}

__global__ void k_keys(const double* __restrict__ re, int64_t n, int dim, int B,
                       double lo0, double lo1, double lo2, double W,
                       uint64_t* __restrict__ keys, int* __restrict__ idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo[3] = {lo0, lo1, lo2};
    const double scale = (double)(1ull << B);
    const double qmax = (double)((1ull << B) - 1ull);
    uint64_t key = 0;
    for (int d = 0; d < dim; ++d) {
        // t = ((x - lo) / W) * 2^B with every operation rounded separately
        double t = __dmul_rn(__ddiv_rn(__dsub_rn(re[i * dim + d], lo[d]), W), scale);
        double qf = floor(t);
        qf = qf < 0.0 ? 0.0 : (qf > qmax ? qmax : qf);
        key |= spread_bits((uint64_t)qf, dim, B) << d;
    }
    keys[i] = key;
    idx[i] = (int)i;
}

__global__ void k_gather_soa(const double* __restrict__ aos, const int* __restrict__ perm, int64_t n,
                             int dim, double* __restrict__ soa) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int d = 0; d < dim; ++d) soa[d * n + i] = aos[j * dim + d];
}

// ---------------------------------------------------------------------------
// box coordinates
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) {
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

__device__ __forceinline__ void decode(uint64_t p, int m, int dim, int64_t* I) {
    for (int d = 0; d < dim; ++d) I[d] = 0;
    for (int b = 0; b < m; ++b)
        for (int d = 0; d < dim; ++d) I[d] |= (int64_t)((p >> (b * dim + d)) & 1ull) << b;
}

__device__ __forceinline__ uint64_t encode(const int64_t* I, int m, int dim) {
    uint64_t p = 0;
    for (int b = 0; b < m; ++b)
        for (int d = 0; d < dim; ++d) p |= (uint64_t)((I[d] >> b) & 1) << (b * dim + d);
    return p;
}

// range of J at level m near box (l, I) on one axis, clamped to the grid
__device__ __forceinline__ void near_range(int l, int64_t I, int m, int k, int64_t* jlo, int64_t* jhi) {
    int f = l > m ? l : m;
    int64_t sb = 1ll << (f - l), sc = 1ll << (f - m);
    int64_t c2 = (2 * I + 1) * sb;
    int64_t lim = (int64_t)k * (sb + sc);
    int64_t lo = -floordiv(-(c2 - lim - sc), 2 * sc);   // ceil
    int64_t hi = floordiv(c2 + lim - sc, 2 * sc);
    int64_t top = (1ll << m) - 1;
    *jlo = lo < 0 ? 0 : lo;
    *jhi = hi > top ? top : hi;
}

__device__ __forceinline__ bool near_boxes(int la, const int64_t* Ia, int lb, const int64_t* Ib, int dim, int k) {
    int f = la > lb ? la : lb;
    int64_t sa = 1ll << (f - la), sb = 1ll << (f - lb);
    int64_t lim = (int64_t)k * (sa + sb);
    for (int d = 0; d < dim; ++d) {
        int64_t diff = (2 * Ia[d] + 1) * sa - (2 * Ib[d] + 1) * sb;
        if (diff > lim || -diff > lim) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// leaves: split passes and level restriction
// ---------------------------------------------------------------------------
struct LeafArrays {   // device arrays in plan scratch
    int* lev = nullptr;
    int* st = nullptr;
    int* en = nullptr;
    uint64_t* pre = nullptr;
    int n = 0;
    void take(int count) {
        Scratch& s = plan_scratch();
        lev = s.take_n<int>(count);
        st = s.take_n<int>(count);
        en = s.take_n<int>(count);
        pre = s.take_n<uint64_t>(count);
        n = count;
    }
};

__device__ __forceinline__ void child_bounds(const uint64_t* __restrict__ keys, int s, int e, uint64_t p,
                                             int level, int dim, int B, int* bnd) {
    // bnd[c] = first index in [s, e) whose level+1 prefix >= (p << dim | c); bnd[2^dim] = e
    int shift = dim * (B - level - 1);
    int nc = 1 << dim;
    for (int c = 0; c < nc; ++c) {
        uint64_t target = (p << dim) | (uint64_t)c;
        int lo = s, hi = e;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if ((keys[mid] >> shift) < target) lo = mid + 1;
            else hi = mid;
        }
        bnd[c] = lo;
    }
    bnd[nc] = e;
}

// mode 0: split when count > Ns or level < force; mode 1: split when flag[i]
__global__ void k_leaf_count(int nl, const int* __restrict__ lev, const uint64_t* __restrict__ pre,
                             const int* __restrict__ st, const int* __restrict__ en,
                             const uint64_t* __restrict__ keys, int dim, int B, int Ns, int force,
                             const int* __restrict__ flag, int* __restrict__ cnt, int* __restrict__ any) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    int l = lev[i];
    bool split = l < B && (flag ? flag[i] != 0 : ((en[i] - st[i]) > Ns || l < force));
    if (!split) {
        cnt[i] = 1;
        return;
    }
    atomicOr(any, 1);
    int bnd[9];
    child_bounds(keys, st[i], en[i], pre[i], l, dim, B, bnd);
    int c = 0;
    for (int j = 0; j < (1 << dim); ++j) c += bnd[j + 1] > bnd[j];
    cnt[i] = c;
}

__global__ void k_leaf_emit(int nl, const int* __restrict__ lev, const uint64_t* __restrict__ pre,
                            const int* __restrict__ st, const int* __restrict__ en,
                            const uint64_t* __restrict__ keys, int dim, int B, int Ns, int force,
                            const int* __restrict__ flag, const int* __restrict__ off,
                            int* __restrict__ olev, uint64_t* __restrict__ opre,
                            int* __restrict__ ost, int* __restrict__ oen) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    int l = lev[i];
    bool split = l < B && (flag ? flag[i] != 0 : ((en[i] - st[i]) > Ns || l < force));
    int o = off[i];
    if (!split) {
        olev[o] = l;
        opre[o] = pre[i];
        ost[o] = st[i];
        oen[o] = en[i];
        return;
    }
    int bnd[9];
    child_bounds(keys, st[i], en[i], pre[i], l, dim, B, bnd);
    for (int j = 0; j < (1 << dim); ++j) {
        if (bnd[j + 1] > bnd[j]) {
            olev[o] = l + 1;
            opre[o] = (pre[i] << dim) | (uint64_t)j;
            ost[o] = bnd[j];
            oen[o] = bnd[j + 1];
            ++o;
        }
    }
}

// box (m, J) exists iff the first leaf starting at or after J's first key lies inside J
// and is at level >= m
__device__ __forceinline__ bool box_exists(int nl, const int* __restrict__ lev, const uint64_t* __restrict__ pre,
                                           int dim, int B, int m, uint64_t q) {
    int sh = dim * (B - m);
    uint64_t ks = q << sh, ke = (q + 1) << sh;
    int lo = 0, hi = nl;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        uint64_t s = pre[mid] << (dim * (B - lev[mid]));
        if (s < ks) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= nl) return false;
    uint64_t s = pre[lo] << (dim * (B - lev[lo]));
    return s < ke && lev[lo] >= m;
}

__global__ void k_balance_flags(int nl, const int* __restrict__ lev, const uint64_t* __restrict__ pre,
                                int dim, int B, int k, int maxl, int* __restrict__ flag, int* __restrict__ any) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    int l = lev[i];
    int m = l + 2;
    int f = 0;
    if (m <= maxl) {
        int64_t I[3], lo[3], hi[3];
        decode(pre[i], l, dim, I);
        for (int d = 0; d < dim; ++d) near_range(l, I[d], m, k, &lo[d], &hi[d]);
        int64_t J[3] = {lo[0], lo[1], dim > 2 ? lo[2] : 0};
        // iterate the window (lexicographic), skipping boxes inside the leaf
        while (!f) {
            bool inside = true;
            for (int d = 0; d < dim; ++d) {
                int64_t r = J[d] - 4 * I[d];
                if (r < 0 || r > 3) inside = false;
            }
            if (!inside && box_exists(nl, lev, pre, dim, B, m, encode(J, m, dim))) f = 1;
            int d = 0;
            for (; d < dim; ++d) {
                if (J[d] < hi[d]) { ++J[d]; break; }
                J[d] = lo[d];
            }
            if (d == dim) break;
        }
    }
    flag[i] = f;
    if (f) atomicOr(any, 1);
}

__global__ void k_leaf_maxlevel(int nl, const int* __restrict__ lev, int* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nl) atomicMax(out, lev[i]);
}

static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

// one split pass; returns true when some leaf was split
static bool split_pass(LeafArrays& L, const uint64_t* keys, int dim, int B, int Ns, int force,
                       const int* flag, cudaStream_t st) {
    int nl = L.n;
    Scratch& scr = plan_scratch();
    int* cnt = scr.take_n<int>(nl);
    int* off = scr.take_n<int>(nl);
    int* any = scr.take_n<int>(1);
    CFMM_CUDA(cudaMemsetAsync(any, 0, sizeof(int), st));
    k_leaf_count<<<blocks_for(nl, 256), 256, 0, st>>>(nl, L.lev, L.pre, L.st, L.en, keys, dim, B, Ns, force, flag,
                                                     cnt, any);
    CFMM_LAUNCHED();
    int64_t total = scan_exclusive(cnt, off, nl, st);
    int h = 0;
    CFMM_CUDA(cudaMemcpyAsync(&h, any, sizeof(int), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    if (!h) return false;
    LeafArrays N;
    N.take((int)total);
    k_leaf_emit<<<blocks_for(nl, 256), 256, 0, st>>>(nl, L.lev, L.pre, L.st, L.en, keys, dim, B, Ns, force, flag,
                                                    off, N.lev, N.pre, N.st, N.en);
    CFMM_LAUNCHED();
    L = N;
    return true;
}

static int leaf_maxlevel(LeafArrays& L, cudaStream_t st) {
    int* m = plan_scratch().take_n<int>(1);
    CFMM_CUDA(cudaMemsetAsync(m, 0, sizeof(int), st));
    k_leaf_maxlevel<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, L.lev, m);
    CFMM_LAUNCHED();
    int h = 0;
    CFMM_CUDA(cudaMemcpyAsync(&h, m, sizeof(int), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    return h;
}

// Leaves in one pass. Repeated splitting (split while a box holds more than Ns
// points or lies above level `force`) puts point i in the box of level
//   l_i = max(min{l : count of the level-l box containing i <= Ns}, force),
// capped at B, since the counts of the boxes containing i do not increase with
// the level; the leaves are the runs of equal (l_i, prefix) in key order, in
// the same (Morton) order as the splitting produces them. base_lev, when
// given, is a per-point lower bound (the level of the point's current leaf).
__global__ void k_pt_level(int64_t n, const uint64_t* __restrict__ keys, int dim, int B, int Ns, int force,
                           const int* __restrict__ base_lev, int* __restrict__ lev) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = keys[i];
    auto count = [&](int l) -> int64_t {
        int sh = dim * (B - l);
        uint64_t p = sh >= 64 ? 0 : (k >> sh);
        uint64_t ks = sh >= 64 ? 0 : (p << sh);
        // first index with key >= ks, first index with key >> sh > p
        int64_t lo = 0, hi = i;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < ks) lo = mid + 1;
            else hi = mid;
        }
        int64_t a = lo;
        lo = i + 1;
        hi = n;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (sh < 64 && (keys[mid] >> sh) <= p) lo = mid + 1;
            else if (sh >= 64) lo = mid + 1;
            else hi = mid;
        }
        return lo - a;
    };
    int l;
    if (base_lev) {
        l = base_lev[i];
    } else {
        // smallest l in [0, B] with count(l) <= Ns (count(B) may still exceed Ns)
        int lo = 0, hi = B;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (count(mid) <= Ns) hi = mid;
            else lo = mid + 1;
        }
        l = lo;
    }
    if (l < force) l = force < B ? force : B;
    lev[i] = l;
}

__global__ void k_pt_from_leaves(int nl, const int* __restrict__ lev, const int* __restrict__ st,
                                 const int* __restrict__ en, int* __restrict__ plev) {
    int j = blockIdx.x;
    for (int i = st[j] + threadIdx.x; i < en[j]; i += blockDim.x) plev[i] = lev[j];
}

__global__ void k_leaf_starts(int64_t n, const uint64_t* __restrict__ keys, int dim, int B,
                              const int* __restrict__ plev, int* __restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f = 1;
    if (i > 0) {
        int l = plev[i], lp = plev[i - 1];
        int sh = dim * (B - l);
        f = !(l == lp && (sh >= 64 || (keys[i] >> sh) == (keys[i - 1] >> sh)));
    }
    flag[i] = f;
}

__global__ void k_leaf_from_pts(int64_t n, const uint64_t* __restrict__ keys, int dim, int B,
                                const int* __restrict__ plev, const int* __restrict__ flag,
                                const int* __restrict__ off, int nl, int* __restrict__ lev,
                                uint64_t* __restrict__ pre, int* __restrict__ st, int* __restrict__ en) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    int j = off[i];
    int l = plev[i];
    int sh = dim * (B - l);
    lev[j] = l;
    pre[j] = sh >= 64 ? 0 : (keys[i] >> sh);
    st[j] = (int)i;
    if (j > 0) en[j - 1] = (int)i;
    if (j == nl - 1) en[j] = (int)n;
}

// leaves of the whole point set (first call: base = null) or of the current
// leaves refined down to level `force` (base = current leaves)
static void refine_onepass(LeafArrays& L, const uint64_t* keys, int64_t n, int dim, int B, int Ns, int force,
                           bool from_current, cudaStream_t st) {
    Scratch& scr = plan_scratch();
    int* plev = scr.take_n<int>(n);
    int* base = nullptr;
    if (from_current) {
        base = scr.take_n<int>(n);
        k_pt_from_leaves<<<L.n, 128, 0, st>>>(L.n, L.lev, L.st, L.en, base);
        CFMM_LAUNCHED();
    }
    k_pt_level<<<blocks_for(n, 256), 256, 0, st>>>(n, keys, dim, B, Ns, force, base, plev);
    CFMM_LAUNCHED();
    int* flag = scr.take_n<int>(n);
    int* off = scr.take_n<int>(n);
    k_leaf_starts<<<blocks_for(n, 256), 256, 0, st>>>(n, keys, dim, B, plev, flag);
    CFMM_LAUNCHED();
    int64_t nl = scan_exclusive(flag, off, (int)n, st);
    LeafArrays N;
    N.take((int)nl);
    k_leaf_from_pts<<<blocks_for(n, 256), 256, 0, st>>>(n, keys, dim, B, plev, flag, off, (int)nl, N.lev, N.pre,
                                                       N.st, N.en);
    CFMM_LAUNCHED();
    L = N;
}

// The deepest leaf level does not change while balancing (only leaves two or
// more levels coarser than a neighbour are split), so it is read once; a split
// pass that splits nothing ends the loop.
static void balance(LeafArrays& L, const uint64_t* keys, int dim, int B, int k, cudaStream_t st) {
    int* any = plan_scratch().take_n<int>(1);
    int maxl = leaf_maxlevel(L, st);
    for (;;) {
        int* flag = plan_scratch().take_n<int>(L.n);
        k_balance_flags<<<blocks_for(L.n, 128), 128, 0, st>>>(L.n, L.lev, L.pre, dim, B, k, maxl, flag, any);
        CFMM_LAUNCHED();
        if (!split_pass(L, keys, dim, B, 0, 0, flag, st)) return;
    }
}

// ---------------------------------------------------------------------------
// boxes from leaves
// ---------------------------------------------------------------------------
// head flags of every level at once: entry m nl + i says whether leaf i
// starts a box of level m (thread per (level, leaf))
__global__ void k_box_flags(int nl, int nlev, const int* __restrict__ lev, const uint64_t* __restrict__ pre,
                            int dim, int* __restrict__ head) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)nl * nlev) return;
    int m = (int)(k / nl), i = (int)(k - (int64_t)m * nl);
    head += (int64_t)m * nl;
    int l = lev[i];
    bool q = l >= m;
    bool h = false;
    if (q) {
        uint64_t pm = pre[i] >> (dim * (l - m));
        if (i == 0) h = true;
        else {
            int lp = lev[i - 1];
            h = lp < m || (pre[i - 1] >> (dim * (lp - m))) != pm;
        }
    }
    head[i] = h ? 1 : 0;
}

// boxes of every level at once (thread per (level, leaf)); idx is the exclusive
// scan of all levels' head flags, level-major, so it counts the boxes of the
// coarser levels too and is the box index itself
__global__ void k_box_emit(int nl, int nlev, const int* __restrict__ lev, const uint64_t* __restrict__ pre,
                           const int* __restrict__ st, const int* __restrict__ en, int dim,
                           const int* __restrict__ head, const int* __restrict__ idx,
                           int* __restrict__ blevel, uint64_t* __restrict__ bpre, int* __restrict__ bst,
                           int* __restrict__ ben, int* __restrict__ bleaf, int* __restrict__ leaf_box) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)nl * nlev) return;
    int m = (int)(k / nl), i = (int)(k - (int64_t)m * nl);
    int l = lev[i];
    if (l < m) return;
    uint64_t pm = pre[i] >> (dim * (l - m));
    int b = idx[k] + head[k] - 1;
    if (head[k]) {
        blevel[b] = m;
        bpre[b] = pm;
        bst[b] = st[i];
        bleaf[b] = (l == m);
        if (l == m) leaf_box[i] = b;
    }
    bool tail;
    if (i == nl - 1) tail = true;
    else {
        int ln = lev[i + 1];
        tail = ln < m || (pre[i + 1] >> (dim * (ln - m))) != pm;
    }
    if (tail) ben[b] = en[i];
}

__device__ __forceinline__ int find_box(const uint64_t* __restrict__ bpre, const int* __restrict__ loff,
                                        int nlev, int m, uint64_t q) {
    if (m < 0 || m >= nlev) return -1;
    int lo = loff[m], hi = loff[m + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (bpre[mid] < q) lo = mid + 1;
        else hi = mid;
    }
    if (lo < loff[m + 1] && bpre[lo] == q) return lo;
    return -1;
}

__device__ __forceinline__ int lower_box(const uint64_t* __restrict__ bpre, int lo, int hi, uint64_t q) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (bpre[mid] < q) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_box_links(int nb, const int* __restrict__ blevel, const uint64_t* __restrict__ bpre,
                            const int* __restrict__ loff, int nlev, int dim, int* __restrict__ parent,
                            int* __restrict__ cbeg, int* __restrict__ cend) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int m = blevel[b];
    uint64_t p = bpre[b];
    parent[b] = m > 0 ? find_box(bpre, loff, nlev, m - 1, p >> dim) : -1;
    if (m + 1 < nlev) {
        int lo = loff[m + 1], hi = loff[m + 2];
        cbeg[b] = lower_box(bpre, lo, hi, p << dim);
        cend[b] = lower_box(bpre, lo, hi, (p + 1) << dim);
    } else {
        cbeg[b] = cend[b] = 0;
    }
}

// per leaf box: sum / min / max of Im x per axis (one warp per box)
__global__ void k_leaf_stats(int nb, const int* __restrict__ bleaf, const int* __restrict__ bst,
                             const int* __restrict__ ben, const double* __restrict__ xi, int64_t n, int dim,
                             double* __restrict__ sum, double* __restrict__ mn, double* __restrict__ mx) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= nb || !bleaf[warp]) return;
    int b = warp;
    for (int d = 0; d < dim; ++d) {
        double s = 0.0, lo = INFINITY, hi = -INFINITY;
        for (int i = bst[b] + lane; i < ben[b]; i += 32) {
            double v = xi[d * n + i];
            s += v;
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            sum[b * dim + d] = s;
            mn[b * dim + d] = lo;
            mx[b * dim + d] = hi;
        }
    }
}

__global__ void k_parent_stats(int lo, int hi, const int* __restrict__ bleaf, const int* __restrict__ cbeg,
                               const int* __restrict__ cend, int dim, double* __restrict__ sum,
                               double* __restrict__ mn, double* __restrict__ mx) {
    int b = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi || bleaf[b]) return;
    for (int d = 0; d < dim; ++d) {
        double s = 0.0, a = INFINITY, z = -INFINITY;
        for (int c = cbeg[b]; c < cend[b]; ++c) {
            s += sum[c * dim + d];
            a = fmin(a, mn[c * dim + d]);
            z = fmax(z, mx[c * dim + d]);
        }
        sum[b * dim + d] = s;
        mn[b * dim + d] = a;
        mx[b * dim + d] = z;
    }
}

__global__ void k_centers(int nb, const int* __restrict__ blevel, const uint64_t* __restrict__ bpre,
                          const int* __restrict__ bst, const int* __restrict__ ben, int dim, double lo0,
                          double lo1, double lo2, double W, const double* __restrict__ sum,
                          double* __restrict__ cre, double* __restrict__ cim) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double lo[3] = {lo0, lo1, lo2};
    int m = blevel[b];
    int64_t I[3];
    decode(bpre[b], m, dim, I);
    double w = ldexp(W, -m);
    double cnt = (double)(ben[b] - bst[b]);
    for (int d = 0; d < dim; ++d) {
        cre[b * dim + d] = lo[d] + ((double)I[d] + 0.5) * w;
        cim[b * dim + d] = sum[b * dim + d] / cnt;
    }
}

// g[m] = max spread over boxes at level m and leaves above m (as uint64 of a non-negative double)
__global__ void k_level_spread(int nb, const int* __restrict__ blevel, const int* __restrict__ bleaf, int nlev,
                               int dim, const double* __restrict__ mn, const double* __restrict__ mx,
                               unsigned long long* __restrict__ g) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double s = 0.0;
    for (int d = 0; d < dim; ++d) s = fmax(s, mx[b * dim + d] - mn[b * dim + d]);
    unsigned long long bits = (unsigned long long)__double_as_longlong(s);
    int m = blevel[b];
    atomicMax(&g[m], bits);
    if (bleaf[b])
        for (int mm = m + 1; mm < nlev; ++mm) atomicMax(&g[mm], bits);
}

// ---------------------------------------------------------------------------
// Lists 1-4 (count, then fill, then sort each box's entries)
// ---------------------------------------------------------------------------
struct ListCtx {
    int nb, nlev, dim, k, l0, B;
    const int* level;
    const int* leaf;
    const int* parent;
    const uint64_t* pre;
    const int* loff;
};

// One warp per box. Candidates of each enumeration window are split over the
// lanes; a ballot keeps the window order, so counts and entries are
// deterministic. Entries are then sorted by box index.
struct Window {
    int m;                  // level of the candidates
    int64_t lo[3], len[3];  // per-axis start and extent
    int64_t total;
};

__device__ __forceinline__ void window_J(const Window& W, int dim, int64_t i, int64_t* J) {
    for (int d = 0; d < dim; ++d) {
        J[d] = W.lo[d] + i % W.len[d];
        i /= W.len[d];
    }
}

// which: 0..3 = List 1..4; out == nullptr counts only. Returns the count (all lanes).
__device__ int list_entries_warp(const ListCtx& C, int which, int b, int* out) {
    const int lane = threadIdx.x & 31;
    int m0 = C.level[b];
    if (m0 < C.l0) return 0;
    int dim = C.dim, k = C.k;
    int64_t I[3];
    decode(C.pre[b], m0, dim, I);
    int cnt = 0;
    // emit helper: every lane holds a candidate result (c or -1)
    auto flush = [&](int c) {
        unsigned mask = __ballot_sync(0xffffffffu, c >= 0);
        if (c >= 0 && out) out[cnt + __popc(mask & ((1u << lane) - 1u))] = c;
        cnt += __popc(mask);
    };
    if (which == 1 && m0 == C.l0) {
        // all boxes of the top level that are not near b
        for (int base = C.loff[m0]; base < C.loff[m0 + 1]; base += 32) {
            int c = base + lane;
            int r = -1;
            if (c < C.loff[m0 + 1]) {
                int64_t J[3];
                decode(C.pre[c], m0, dim, J);
                if (!near_boxes(m0, I, m0, J, dim, k)) r = c;
            }
            flush(r);
        }
        return cnt;
    }
    if (which == 0 && !C.leaf[b]) return 0;
    if (which == 2 && !C.leaf[b]) return 0;
    if (which == 3 && m0 < 1) return 0;
    // windows per list
    int mlo, mhi;
    if (which == 0) { mlo = m0 - 1; mhi = m0 + 1; }
    else if (which == 1) { mlo = mhi = m0; }
    else if (which == 2) { mlo = m0 + 1; mhi = m0 + 2; }
    else { mlo = m0 - 2; mhi = m0 - 1; }
    for (int m = mlo; m <= mhi; ++m) {
        if (m < 0 || m >= C.nlev) continue;
        if (which == 3 && m < C.l0) continue;
        Window w;
        w.m = m;
        w.total = 1;
        bool empty = false;
        for (int d = 0; d < dim; ++d) {
            int64_t lo, hi;
            if (which == 0) {
                near_range(m0, I[d], m, k, &lo, &hi);
            } else if (which == 1) {
                int64_t ip = I[d] >> 1, top = (1ll << m0) - 1;
                lo = 2 * (ip - k);
                hi = 2 * (ip + k) + 1;
                lo = lo < 0 ? 0 : lo;
                hi = hi > top ? top : hi;
            } else if (which == 2) {
                int64_t plo, phi;
                near_range(m0, I[d], m - 1, k, &plo, &phi);
                lo = 2 * plo;
                hi = 2 * phi + 1;
            } else {
                near_range(m0 - 1, I[d] >> 1, m, k, &lo, &hi);
            }
            if (hi < lo) empty = true;
            w.lo[d] = lo;
            w.len[d] = hi - lo + 1;
            w.total *= empty ? 0 : w.len[d];
        }
        if (empty) continue;
        for (int64_t base = 0; base < w.total; base += 32) {
            int64_t i = base + lane;
            int r = -1;
            if (i < w.total) {
                int64_t J[3];
                window_J(w, dim, i, J);
                bool ok = true;
                if (which == 1 || which == 2 || which == 3) ok = !near_boxes(m0, I, m, J, dim, k);
                if (ok) {
                    int c = find_box(C.pre, C.loff, C.nlev, m, encode(J, m, dim));
                    if (c >= 0 && (which == 0 || which == 3 ? C.leaf[c] != 0 : true)) r = c;
                }
            }
            flush(r);
        }
    }
    return cnt;
}

__global__ void k_list_count(ListCtx C, int which, int* __restrict__ cnt) {
    int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= C.nb) return;
    int c = C.nb == 1 ? (which == 0 ? 1 : 0) : list_entries_warp(C, which, b, nullptr);
    if ((threadIdx.x & 31) == 0) cnt[b] = c;
}

__global__ void k_list_fill(ListCtx C, int which, const int* __restrict__ off, int* __restrict__ ent) {
    int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= C.nb) return;
    int* out = ent + off[b];
    if (C.nb == 1) {
        if (which == 0 && (threadIdx.x & 31) == 0) out[0] = 0;
        return;
    }
    int c = list_entries_warp(C, which, b, out);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        // insertion sort by box index (windows are enumerated in coordinate order)
        for (int i = 1; i < c; ++i) {
            int v = out[i], j = i - 1;
            while (j >= 0 && out[j] > v) {
                out[j + 1] = out[j];
                --j;
            }
            out[j + 1] = v;
        }
    }
}

// P2P work: sum over leaves of n_t * sum_{List 1} n_s
__global__ void k_p2p_work(int nb, const int* __restrict__ off, const int* __restrict__ ent,
                           const int* __restrict__ bst, const int* __restrict__ ben,
                           unsigned long long* __restrict__ acc) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    unsigned long long s = 0;
    for (int j = off[b]; j < off[b + 1]; ++j) s += (unsigned long long)(ben[ent[j]] - bst[ent[j]]);
    s *= (unsigned long long)(ben[b] - bst[b]);
    if (s) atomicAdd(acc, s);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
// boxes at levels <= m (cumulative over the level-major scan)
__global__ void k_level_totals(int nlev, int nl, const int* __restrict__ head, const int* __restrict__ idx,
                               int* __restrict__ tot) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < nlev) tot[m] = idx[(int64_t)m * nl + nl - 1] + head[(int64_t)m * nl + nl - 1];
}

static void build_boxes(cfmm_plan_s* P, LeafArrays& L, cudaStream_t st) {
    TreeDev& T = P->tree;
    int dim = P->dim;
    int maxl = leaf_maxlevel(L, st);
    int nl = L.n;
    int nlev = maxl + 1;
    Scratch& scr = plan_scratch();
    int* head = scr.take_n<int>((size_t)nlev * nl);
    int* idx = scr.take_n<int>((size_t)nlev * nl);
    int* leaf_box = scr.take_n<int>(nl);
    int* tot = scr.take_n<int>(nlev);
    // head flags of every level, one level-major scan, then all totals in one read
    int64_t nall = (int64_t)nlev * nl;
    k_box_flags<<<(unsigned)((nall + 255) / 256), 256, 0, st>>>(nl, nlev, L.lev, L.pre, dim, head);
    CFMM_LAUNCHED();
    scan_exclusive_async(head, idx, (int)nall, st);
    k_level_totals<<<blocks_for(nlev, 64), 64, 0, st>>>(nlev, nl, head, idx, tot);
    CFMM_LAUNCHED();
    std::vector<int> cum(nlev);
    CFMM_CUDA(cudaMemcpyAsync(cum.data(), tot, sizeof(int) * nlev, cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    T.nlevels = nlev;
    T.level_off.assign(T.nlevels + 1, 0);
    for (int m = 0; m <= maxl; ++m) T.level_off[m + 1] = cum[m];
    T.nboxes = T.level_off[T.nlevels];
    T.nleaves = nl;
    int nb = T.nboxes;
    T.level.alloc(nb);
    T.prefix.alloc(nb);
    T.start.alloc(nb);
    T.end.alloc(nb);
    T.leaf.alloc(nb);
    T.parent.alloc(nb);
    T.cbeg.alloc(nb);
    T.cend.alloc(nb);
    k_box_emit<<<(unsigned)((nall + 255) / 256), 256, 0, st>>>(nl, nlev, L.lev, L.pre, L.st, L.en, dim, head, idx,
                                                               T.level.get(), T.prefix.get(), T.start.get(),
                                                               T.end.get(), T.leaf.get(), leaf_box);
    CFMM_LAUNCHED();
    T.d_level_off.alloc(T.nlevels + 1);
    upload(T.d_level_off.get(), T.level_off.data(), sizeof(int) * (T.nlevels + 1), st);
    k_box_links<<<blocks_for(nb, 256), 256, 0, st>>>(nb, T.level.get(), T.prefix.get(), T.d_level_off.get(),
                                                    T.nlevels, dim, T.parent.get(), T.cbeg.get(), T.cend.get());
    CFMM_LAUNCHED();
    T.leaf_boxes.resize(nl);
    CFMM_CUDA(cudaMemcpyAsync(T.leaf_boxes.data(), leaf_box, sizeof(int) * nl, cudaMemcpyDeviceToHost, st));
    T.d_leaf_boxes.alloc(nl);
    CFMM_CUDA(cudaMemcpyAsync(T.d_leaf_boxes.get(), leaf_box, sizeof(int) * nl, cudaMemcpyDeviceToDevice, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
}

// per-box Im statistics; fills centres and (optionally) the per-level spread
static void box_stats(cfmm_plan_s* P, cudaStream_t st, std::vector<double>* spread) {
    TreeDev& T = P->tree;
    int dim = P->dim, nb = T.nboxes;
    Scratch& scr = plan_scratch();
    double* sum = scr.take_n<double>((size_t)nb * dim);
    double* mn = scr.take_n<double>((size_t)nb * dim);
    double* mx = scr.take_n<double>((size_t)nb * dim);
    k_leaf_stats<<<blocks_for((int64_t)nb * 32, 256), 256, 0, st>>>(nb, T.leaf.get(), T.start.get(), T.end.get(),
                                                                   P->xi.get(), P->n, dim, sum, mn, mx);
    CFMM_LAUNCHED();
    for (int m = T.nlevels - 2; m >= 0; --m) {
        int lo = T.level_off[m], hi = T.level_off[m + 1];
        k_parent_stats<<<blocks_for(hi - lo, 128), 128, 0, st>>>(lo, hi, T.leaf.get(), T.cbeg.get(), T.cend.get(),
                                                                dim, sum, mn, mx);
        CFMM_LAUNCHED();
    }
    T.cen_re.alloc((size_t)nb * dim);
    T.cen_im.alloc((size_t)nb * dim);
    k_centers<<<blocks_for(nb, 256), 256, 0, st>>>(nb, T.level.get(), T.prefix.get(), T.start.get(), T.end.get(), dim,
                                                  P->lo[0], P->lo[1], P->lo[2], P->W, sum, T.cen_re.get(),
                                                  T.cen_im.get());
    CFMM_LAUNCHED();
    if (spread) {
        unsigned long long* g = scr.take_n<unsigned long long>(T.nlevels);
        CFMM_CUDA(cudaMemsetAsync(g, 0, sizeof(unsigned long long) * T.nlevels, st));
        k_level_spread<<<blocks_for(nb, 256), 256, 0, st>>>(nb, T.level.get(), T.leaf.get(), T.nlevels, dim,
                                                           mn, mx, g);
        CFMM_LAUNCHED();
        std::vector<unsigned long long> h(T.nlevels);
        CFMM_CUDA(cudaMemcpyAsync(h.data(), g, sizeof(unsigned long long) * T.nlevels,
                                  cudaMemcpyDeviceToHost, st));
        CFMM_CUDA(cudaStreamSynchronize(st));
        spread->resize(T.nlevels);
        for (int m = 0; m < T.nlevels; ++m) {
            double v;
            memcpy(&v, &h[m], sizeof(double));
            (*spread)[m] = v;
        }
    }
    CFMM_CUDA(cudaStreamSynchronize(st));
}

static void build_lists(cfmm_plan_s* P, cudaStream_t st) {
    TreeDev& T = P->tree;
    int nb = T.nboxes;
    ListCtx C{nb, T.nlevels, P->dim, P->sep, T.l0, P->B, T.level.get(), T.leaf.get(), T.parent.get(),
              T.prefix.get(), T.d_level_off.get()};
    // counts and scans of the four lists, then one read of the four totals
    int* cnt = plan_scratch().take_n<int>((size_t)4 * (nb + 1));
    for (int w = 0; w < 4; ++w) {
        int* cw = cnt + (size_t)w * (nb + 1);
        k_list_count<<<blocks_for((int64_t)nb * 32, 128), 128, 0, st>>>(C, w, cw);
        CFMM_LAUNCHED();
        CFMM_CUDA(cudaMemsetAsync(cw + nb, 0, sizeof(int), st));
        T.loff[w].alloc(nb + 1);
        scan_exclusive_async(cw, T.loff[w].get(), nb + 1, st);   // loff[nb] = total
    }
    // the four offset arrays come back to the host in one read (the setup of
    // the expansions walks them there)
    int tot[4];
    for (int w = 0; w < 4; ++w) {
        T.hloff[w].resize(nb + 1);
        CFMM_CUDA(cudaMemcpyAsync(T.hloff[w].data(), T.loff[w].get(), sizeof(int) * (nb + 1),
                                  cudaMemcpyDeviceToHost, st));
    }
    CFMM_CUDA(cudaStreamSynchronize(st));
    for (int w = 0; w < 4; ++w) {
        tot[w] = T.hloff[w][nb];
        CFMM_REQUIRE(tot[w] >= 0, CFMM_EUNSUPPORTED, "interaction list longer than 2^31 entries");
        T.llen[w] = tot[w];
        T.lent[w].alloc(tot[w] > 0 ? tot[w] : 1);
        k_list_fill<<<blocks_for((int64_t)nb * 32, 128), 128, 0, st>>>(C, w, T.loff[w].get(), T.lent[w].get());
        CFMM_LAUNCHED();
    }
    // work counters
    unsigned long long* acc = plan_scratch().take_n<unsigned long long>(1);
    CFMM_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st));
    k_p2p_work<<<blocks_for(nb, 256), 256, 0, st>>>(nb, T.loff[0].get(), T.lent[0].get(), T.start.get(),
                                                   T.end.get(), acc);
    CFMM_LAUNCHED();
    unsigned long long h = 0;
    CFMM_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    P->p2p_pairs = (int64_t)h;
    P->m2l_pairs = T.llen[1];
}

// Builds the sorted geometry and the tree of a plan. re/im (and nre/nim when
// not null) are device copies of the caller's [n][dim] arrays.
// Lipschitz estimate of Im x against Re x (Assumptions 4.1/5.1): over the
// pairs of points at most kLipWindow apart in Morton order (spatially close),
// max |Im(x_i - x_j)|^2 / |Re(x_i - x_j)|^2, as the bits of a non-negative
// float (inf when Re x_i = Re x_j but Im x_i != Im x_j). Coincident points
// are skipped.
constexpr int kLipWindow = 32;
constexpr int kLipBlock = 256;
__global__ void __launch_bounds__(kLipBlock) k_lipschitz(const double* __restrict__ xr, const double* __restrict__ xi,
                                                         int64_t n, int dim, unsigned* __restrict__ out) {
    // the block's points and the kLipWindow after them (differences in FP64,
    // their squares in FP32: the ratio needs no more precision)
    __shared__ double sre[3][kLipBlock + kLipWindow], sim[3][kLipBlock + kLipWindow];
    __shared__ unsigned best_s;
    int64_t i0 = blockIdx.x * (int64_t)kLipBlock;
    if (threadIdx.x == 0) best_s = 0u;
    for (int k = threadIdx.x; k < kLipBlock + kLipWindow; k += blockDim.x) {
        int64_t j = i0 + k;
        for (int a = 0; a < dim; ++a) {
            sre[a][k] = j < n ? xr[a * n + j] : 0.0;
            sim[a][k] = j < n ? xi[a * n + j] : 0.0;
        }
    }
    __syncthreads();
    int t = threadIdx.x;
    int64_t i = i0 + t;
    float best = 0.f;
    if (i < n) {
        int cnt = (int)min((int64_t)kLipWindow, n - 1 - i);
        for (int q = 1; q <= cnt; ++q) {
            float a2 = 0.f, b2 = 0.f;
            for (int a = 0; a < dim; ++a) {
                float dr = (float)(sre[a][t] - sre[a][t + q]), di = (float)(sim[a][t] - sim[a][t + q]);
                a2 = fmaf(dr, dr, a2);
                b2 = fmaf(di, di, b2);
            }
            if (b2 == 0.f) continue;
            best = fmaxf(best, a2 > 0.f ? b2 / a2 : INFINITY);
        }
    }
    atomicMax(&best_s, __float_as_uint(best));
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(out, best_s);
}

// Largest Lipschitz constant L for which the Sec. 6.3 criterion C_L r/R < 1
// holds at separation k (R = (k + 1/2) w, r = sqrt(d)/2 w): 2D C_L =
// (1+L)/(1-L) (Eq. nterms_criteria_2d), 3D C_L = sqrt(L^2+10L+1)/(1-L)
// (Eqs. eta_const, nterms_criteria_3d).
static double lipschitz_limit(int dim, int k) {
    double c = (k + 0.5) / (std::sqrt((double)dim) * 0.5);
    if (dim == 2) return (c - 1.0) / (c + 1.0);
    // L^2 + 10 L + 1 = c^2 (1 - L)^2, root in (0, 1)
    double a = 1.0 - c * c, b = 10.0 + 2.0 * c * c, q = 1.0 - c * c;
    double disc = std::sqrt(b * b - 4.0 * a * q);
    double r1 = (-b + disc) / (2.0 * a), r2 = (-b - disc) / (2.0 * a);
    return (r1 > 0.0 && r1 < 1.0) ? r1 : r2;
}

// automatic separation: the smallest k in 1..3 with kSepLipFactor * limit(k) >= L
// (kSepLipFactor calibrated on the surface and curve workloads; 3 if none)
constexpr double kSepLipFactor = 2.0;
int auto_separation(int dim, double L) {
    for (int k = 1; k <= 3; ++k)
        if (kSepLipFactor * lipschitz_limit(dim, k) >= L) return k;
    return 3;
}

void build_tree(cfmm_plan_s* P, const double* re, const double* im, const double* nre, const double* nim,
                int top_level_opt) {
    cudaStream_t st = P->stream;
    int dim = P->dim;
    int64_t n = P->n;
    PhaseTimer pt(st);
    // finite check
    {
        int* flag = plan_scratch().take_n<int>(1);
        CFMM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
        int g = blocks_for(n * dim, 256);
        g = g > 4096 ? 4096 : g;
        k_nonfinite<<<g, 256, 0, st>>>(re, n * dim, flag);
        k_nonfinite<<<g, 256, 0, st>>>(im, n * dim, flag);
        ::cfmm::count_launch(2);
        if (nre) {
            k_nonfinite<<<g, 256, 0, st>>>(nre, n * dim, flag);
            k_nonfinite<<<g, 256, 0, st>>>(nim, n * dim, flag);
            ::cfmm::count_launch(2);
        }
        CFMM_CUDA(cudaGetLastError());
        int h = 0;
        CFMM_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        CFMM_CUDA(cudaStreamSynchronize(st));
        CFMM_REQUIRE(h == 0, CFMM_ENONFINITE, "points or normals contain NaN or Inf");
    }
    // a1: bounding square (Sec. 6.1)
    {
        int nblk = blocks_for(n, 256);
        nblk = nblk > 1024 ? 1024 : nblk;
        double* part = plan_scratch().take_n<double>((size_t)nblk * 2 * dim);
        k_bbox<<<nblk, 256, 0, st>>>(re, n, dim, part);
        CFMM_LAUNCHED();
        std::vector<double> h((size_t)nblk * 2 * dim);
        CFMM_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
        CFMM_CUDA(cudaStreamSynchronize(st));
        double mn[3], mx[3];
        for (int d = 0; d < dim; ++d) {
            mn[d] = INFINITY;
            mx[d] = -INFINITY;
        }
        for (int b = 0; b < nblk; ++b)
            for (int d = 0; d < dim; ++d) {
                mn[d] = std::min(mn[d], h[b * 2 * dim + d]);
                mx[d] = std::max(mx[d], h[b * 2 * dim + dim + d]);
            }
        double ext = 0.0;
        for (int d = 0; d < dim; ++d) ext = std::max(ext, mx[d] - mn[d]);
        double W = ext * (1.0 + std::ldexp(1.0, -20));
        if (W == 0.0) W = 1.0;
        P->W = W;
        for (int d = 0; d < 3; ++d) P->lo[d] = 0.0;
        for (int d = 0; d < dim; ++d) {
            double c = (mn[d] + mx[d]) * 0.5;
            P->lo[d] = c - W * 0.5;
        }
    }
    pt.mark("check+bbox");
    // a2: keys, stable radix sort, gather
    P->B = dim == 2 ? 31 : 21;
    int B = P->B;
    P->keys.alloc(n);
    P->perm.alloc(n);
    k_keys<<<blocks_for(n, 256), 256, 0, st>>>(re, n, dim, B, P->lo[0], P->lo[1], P->lo[2], P->W, P->keys.get(),
                                              P->perm.get());
    CFMM_LAUNCHED();
    radix_sort(P->keys, P->perm, (int)n, dim * B, st);
    P->xr.alloc((size_t)n * dim);
    P->xi.alloc((size_t)n * dim);
    k_gather_soa<<<blocks_for(n, 256), 256, 0, st>>>(re, P->perm.get(), n, dim, P->xr.get());
    k_gather_soa<<<blocks_for(n, 256), 256, 0, st>>>(im, P->perm.get(), n, dim, P->xi.get());
    ::cfmm::count_launch(2);
    if (nre) {
        P->nr.alloc((size_t)n * dim);
        P->ni.alloc((size_t)n * dim);
        k_gather_soa<<<blocks_for(n, 256), 256, 0, st>>>(nre, P->perm.get(), n, dim, P->nr.get());
        k_gather_soa<<<blocks_for(n, 256), 256, 0, st>>>(nim, P->perm.get(), n, dim, P->ni.get());
        ::cfmm::count_launch(2);
    }
    CFMM_CUDA(cudaGetLastError());
    pt.mark("keys+sort");
    // geometry assumption: Re r^2 > 0 for close pairs (Lipschitz estimate < 1)
    {
        unsigned* d = plan_scratch().take_n<unsigned>(1);
        CFMM_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned), st));
        if (n > 1) {
            k_lipschitz<<<blocks_for(n, kLipBlock), kLipBlock, 0, st>>>(P->xr.get(), P->xi.get(), n, dim, d);
            CFMM_LAUNCHED();
        }
        unsigned h = 0;
        CFMM_CUDA(cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CFMM_CUDA(cudaStreamSynchronize(st));
        float r;
        std::memcpy(&r, &h, sizeof(float));
        P->lipschitz = std::sqrt((double)r);
        CFMM_REQUIRE(P->lipschitz < 1.0, CFMM_EGEOM,
                     "geometry outside the method's assumptions: Re r^2 <= 0 for a close pair (|Im dx| >= |Re dx|)");
        if (P->sep <= 0) P->sep = auto_separation(dim, P->lipschitz);
    }
    pt.mark("lipschitz");
    // a3: leaves, level restriction
    LeafArrays L;
    L.take(1);
    {
        // the root leaf: level 0, prefix 0, points [0, n)
        int z = 0, nn = (int)n;
        uint64_t zp = 0;
        upload(L.lev, &z, sizeof(int), st);
        upload(L.pre, &zp, sizeof(uint64_t), st);
        upload(L.st, &z, sizeof(int), st);
        upload(L.en, &nn, sizeof(int), st);
    }
    int Ns = P->leaf_size;
    refine_onepass(L, P->keys.get(), n, dim, B, Ns, 0, false, st);
    pt.mark("refine");
    balance(L, P->keys.get(), dim, B, P->sep, st);
    pt.mark("balance");
    build_boxes(P, L, st);
    pt.mark("boxes");
    // a4 + top expansion level
    std::vector<double> spread;
    bool helm = P->kernel == CFMM_HELMHOLTZ;
    box_stats(P, st, (helm && n > Ns && top_level_opt <= 0) ? &spread : nullptr);
    int l0 = 1;
    if (n > Ns) {
        if (top_level_opt > 0) {
            l0 = top_level_opt;
        } else if (helm) {
            // tau = c_d ln(eps / 2^-52), c_2 = 1, c_3 = 2 (calibrated on the 2D curve
            // and 3D surface workloads): the coarsest level whose boxes (and coarser
            // leaves) have kappa sqrt(d) g <= tau; below the deepest level the spread
            // is taken to halve per level (Im x Lipschitz in Re x)
            double tau = (dim == 2 ? 1.0 : 2.0) * std::log(P->eps / std::ldexp(1.0, -52));
            int maxl = P->tree.nlevels - 1;
            double sq = std::sqrt((double)dim);
            l0 = 0;
            for (int m = 1; m <= maxl; ++m)
                if (P->kappa * sq * spread[m] <= tau) {
                    l0 = m;
                    break;
                }
            if (l0 == 0) {
                int m = maxl < 1 ? 1 : maxl;
                double gm = maxl < 1 ? 0.0 : spread[maxl];
                while (m < B && P->kappa * sq * gm > tau) {
                    ++m;
                    gm *= 0.5;
                }
                l0 = m;
            }
            // CFMM_TOP_FIT: deeper while the 3D order at l0 exceeds the limit of
            // the translation kernels (the order falls with the box width)
            if (top_level_opt == -1 && dim == 3)
                while (l0 < B && nterms_helm3d(P->sep, P->eps * 0.01, P->kappa, std::ldexp(P->W, -l0)) > kMaxP3Top)
                    ++l0;
        }
        // boxes are stored level-major, so the leaf with the smallest box index
        // is the coarsest; when no leaf lies above l0 the forced refinement
        // and the re-balancing change nothing and are skipped
        int min_leaf_level = P->tree.nlevels;
        if (!P->tree.leaf_boxes.empty()) {
            int bmin = *std::min_element(P->tree.leaf_boxes.begin(), P->tree.leaf_boxes.end());
            min_leaf_level = (int)(std::upper_bound(P->tree.level_off.begin(), P->tree.level_off.end(), bmin) -
                                   P->tree.level_off.begin()) - 1;
        }
        if (l0 > 1 && min_leaf_level < l0) {
            refine_onepass(L, P->keys.get(), n, dim, B, Ns, l0, true, st);
            balance(L, P->keys.get(), dim, B, P->sep, st);
            build_boxes(P, L, st);
            box_stats(P, st, nullptr);
        }
    }
    P->tree.l0 = l0;
    pt.mark("centres+l0");
}

// a5: Lists 1-4 of the plan's tree (after build_tree)
void build_plan_lists(cfmm_plan_s* P) {
    PhaseTimer pt(P->stream);
    build_lists(P, P->stream);
    pt.mark("lists");
}

}  // namespace cfmm
