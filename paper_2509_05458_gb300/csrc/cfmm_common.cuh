// Common definitions of the CUDA path: complex arithmetic, status handling,
// launch accounting and the plan object.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../include/cfmm.h"

#define CFMM_HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------------------
// complex128 / complex64 value types (interleaved re, im)
// ---------------------------------------------------------------------------
struct cd {
    double x, y;
};
struct cf {
    float x, y;
};

CFMM_HD cd mk(double a, double b) { return cd{a, b}; }
CFMM_HD cd operator+(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
CFMM_HD cd operator-(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
CFMM_HD cd operator-(cd a) { return cd{-a.x, -a.y}; }
CFMM_HD cd operator*(cd a, cd b) { return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
CFMM_HD cd operator*(double s, cd a) { return cd{s * a.x, s * a.y}; }
CFMM_HD cd operator*(cd a, double s) { return cd{s * a.x, s * a.y}; }
CFMM_HD cd& operator+=(cd& a, cd b) { a.x += b.x; a.y += b.y; return a; }
// acc + a b as four fused multiply-adds (the operators above cost two more
// FP64 instructions: the product is rounded before it is added)
CFMM_HD cd cmac(cd acc, cd a, cd b) {
    return cd{fma(-a.y, b.y, fma(a.x, b.x, acc.x)), fma(a.y, b.x, fma(a.x, b.y, acc.y))};
}
// acc + s z for real s (two fused multiply-adds)
CFMM_HD cd rmac(cd acc, double s, cd z) { return cd{fma(s, z.x, acc.x), fma(s, z.y, acc.y)}; }
CFMM_HD cd& operator-=(cd& a, cd b) { a.x -= b.x; a.y -= b.y; return a; }
CFMM_HD double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
CFMM_HD cd conjg(cd a) { return cd{a.x, -a.y}; }
CFMM_HD cd mul_i(cd a) { return cd{-a.y, a.x}; }   // i * a
// a / b with scaling against overflow (Smith's method)
CFMM_HD cd operator/(cd a, cd b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return cd{(a.x + a.y * r) / den, (a.y - a.x * r) / den};
    } else {
        double r = b.x / b.y, den = b.x * r + b.y;
        return cd{(a.x * r + a.y) / den, (a.y * r - a.x) / den};
    }
}
CFMM_HD cd operator/(cd a, double s) { return cd{a.x / s, a.y / s}; }
CFMM_HD cd cinv(cd b) { return cd{1.0, 0.0} / b; }

CFMM_HD cf mkf(float a, float b) { return cf{a, b}; }
CFMM_HD cf operator+(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
CFMM_HD cf operator-(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
CFMM_HD cf operator*(cf a, cf b) { return cf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
CFMM_HD cf operator*(float s, cf a) { return cf{s * a.x, s * a.y}; }
CFMM_HD cf operator-(cf a) { return cf{-a.x, -a.y}; }
CFMM_HD cf cinvf(cf b) {
    float den = b.x * b.x + b.y * b.y;
    return cf{b.x / den, -b.y / den};
}
CFMM_HD cf csqrtf_p(cf z) {
    float a = z.x, b = z.y;
    if (a == 0.f && b == 0.f) return cf{0.f, 0.f};
    float m = hypotf(a, b);
    float t = sqrtf(0.5f * (fabsf(a) + m));
    if (a >= 0.f) return cf{t, b / (2.f * t)};
    return cf{fabsf(b) / (2.f * t), copysignf(t, b)};
}
CFMM_HD cf mul_if(cf a) { return cf{-a.y, a.x}; }   // i * a
// acc + a b as four fused multiply-adds
CFMM_HD cf cmacf(cf acc, cf a, cf b) {
    return cf{fmaf(-a.y, b.y, fmaf(a.x, b.x, acc.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, acc.y))};
}
CFMM_HD cf to_cf(cd a) { return cf{(float)a.x, (float)a.y}; }

// Compensated (Kahan) complex64 sum; value() returns it in complex128
struct Kahan {
    float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
    CFMM_HD void add(cf v) {
        float yx = v.x - cx, tx = sx + yx;
        cx = (tx - sx) - yx;
        sx = tx;
        float yy = v.y - cy, ty = sy + yy;
        cy = (ty - sy) - yy;
        sy = ty;
    }
    CFMM_HD cd value() const { return cd{(double)sx - (double)cx, (double)sy - (double)cy}; }
};

// ---------------------------------------------------------------------------
// status + launch accounting
// ---------------------------------------------------------------------------
namespace cfmm {

void set_error(int status, const std::string& msg);
std::atomic<int64_t>& launch_counter();

inline void count_launch(int n = 1) { launch_counter().fetch_add(n, std::memory_order_relaxed); }

struct Error {
    int status;
    std::string msg;
};

#define CFMM_CUDA(call)                                                              \
    do {                                                                             \
        cudaError_t e__ = (call);                                                    \
        if (e__ != cudaSuccess) {                                                    \
            throw ::cfmm::Error{e__ == cudaErrorMemoryAllocation ? CFMM_ENOMEM       \
                                                                  : CFMM_ECUDA,      \
                                std::string(#call) + ": " + cudaGetErrorString(e__)}; \
        }                                                                            \
    } while (0)

#define CFMM_LAUNCHED()                                                              \
    do {                                                                             \
        ::cfmm::count_launch();                                                      \
        cudaError_t e__ = cudaGetLastError();                                        \
        if (e__ != cudaSuccess)                                                      \
            throw ::cfmm::Error{CFMM_ECUDA, std::string("launch: ") + cudaGetErrorString(e__)}; \
    } while (0)

#define CFMM_REQUIRE(cond, status, msg)                                              \
    do {                                                                             \
        if (!(cond)) throw ::cfmm::Error{status, msg};                               \
    } while (0)

// Caching device allocator (api.cu): blocks freed by plans are kept in
// per-device size classes and handed out again, so plan construction and
// destruction make no cudaMalloc/cudaFree calls in steady state.
void* pool_alloc(size_t bytes, int* dev_out);
void pool_free(void* p, size_t bytes, int dev);

// owning device buffer (memory from the caching allocator). Growing a buffer
// that may still be read by queued work synchronises the device first, as the
// cudaFree it replaces did; plans synchronise their stream before they free.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    int dev = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) pool_free(p, (n ? n : 1) * sizeof(T), dev);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        if (count <= n && p) return;
        if (p) {
            cudaDeviceSynchronize();
            release();
        }
        size_t bytes = (count ? count : 1) * sizeof(T);
        p = (T*)pool_alloc(bytes, &dev);
        n = count;
    }
    T* get() const { return p; }
};

// Bump allocator over cached device chunks for the temporaries of plan
// construction (one per host thread and device). take() never frees; rewind()
// makes the memory reusable once the work that used it has completed.
class Scratch {
   public:
    void* take(size_t bytes);
    template <class T>
    T* take_n(size_t n) {
        return static_cast<T*>(take((n ? n : 1) * sizeof(T)));
    }
    void rewind() {
        cur_ = 0;
        off_ = 0;
    }
    ~Scratch();

   private:
    struct Chunk {
        char* p;
        size_t size;
    };
    std::vector<Chunk> chunks_;
    size_t cur_ = 0, off_ = 0;
};
Scratch& plan_scratch();

// Pinned host staging for the small uploads of plan construction: a copy from
// pinned memory is asynchronous, one from pageable memory costs the host a
// staging copy each time. Bump-allocated like Scratch and rewound with it,
// after the plan's stream has been synchronised.
class HostStage {
   public:
    void* take(size_t bytes);
    void rewind() {
        cur_ = 0;
        off_ = 0;
    }
    ~HostStage();

   private:
    struct Chunk {
        char* p;
        size_t size;
    };
    std::vector<Chunk> chunks_;
    size_t cur_ = 0, off_ = 0;
};
HostStage& plan_host_stage();

// Phase times of plan construction on stderr when CFMM_PLAN_PROFILE=1 (each
// mark synchronises the stream first; off otherwise)
struct PhaseTimer {
    bool on;
    cudaStream_t st;
    std::chrono::steady_clock::time_point t;
    explicit PhaseTimer(cudaStream_t s) : st(s) {
        const char* e = getenv("CFMM_PLAN_PROFILE");
        on = e && e[0] == '1';
        t = std::chrono::steady_clock::now();
    }
    void mark(const char* name) {
        if (!on) return;
        cudaStreamSynchronize(st);
        auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[cfmm plan] %-14s %8.3f ms\n", name,
                std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

// host -> device copy of `bytes` on `st` through the plan's pinned staging
void upload(void* dst, const void* src, size_t bytes, cudaStream_t st);

// ---------------------------------------------------------------------------
// constants shared by host and device code of this library
// ---------------------------------------------------------------------------
constexpr int kMaxDim = 3;
constexpr int kLagNodes = 24;       // Gauss-Laguerre nodes for Hankel functions
constexpr double kHankelSeriesMax = 6.0;  // |z| at or below: ascending series

// Gauss-Laguerre rules for weights u^{-1/2} e^{-u} (rule 0) and u^{1/2} e^{-u}
// (rule 1), built on the host at library load (Golub-Welsch) and copied to
// device constant memory.
struct LagRule {
    double x[2][kLagNodes];
    double w[2][kLagNodes];
};
const LagRule& host_lag_rule();
void ensure_device_tables();   // per device, idempotent

// Tree and list storage of a plan (device pointers unless noted).
struct TreeDev {
    int nboxes = 0, nlevels = 0, nleaves = 0, l0 = 1;
    std::vector<int> level_off;     // host copy [nlevels+1]
    DevBuf<int> d_level_off;
    DevBuf<int> level, start, end, parent, cbeg, cend, leaf;
    DevBuf<uint64_t> prefix;
    DevBuf<double> cen_re, cen_im;  // [nboxes][dim]
    DevBuf<int> loff[4];            // CSR offsets [nboxes+1]
    std::vector<int> hloff[4];      // host copies of the offsets
    DevBuf<int> lent[4];            // CSR entries
    int64_t llen[4] = {0, 0, 0, 0};
    std::vector<int> leaf_boxes;    // host: box index of every leaf, Morton order
    DevBuf<int> d_leaf_boxes;
};

}  // namespace cfmm

struct cfmm_plan_s {
    int dim = 2, kernel = 0, flags = 0, sep = 1, leaf_size = 64, precision = 0;
    bool slp = true, dlp = false, green = false;
    double kappa = 0.0, eps = 1e-6;
    int64_t n = 0;                   // points of the tree (sources + separate targets)
    int64_t n_src = 0;               // caller's sources: union indices [0, n_src)
    int64_t n_trg = 0;               // separate targets: union indices [n_src, n); 0 = targets are the sources
    cudaStream_t stream = nullptr;
    int device = 0;
    double lo[3] = {0, 0, 0};
    double W = 1.0;
    int B = 31;
    double lipschitz = 0.0;          // estimate of the Lipschitz constant of Im x against Re x
    // sorted geometry (SoA [dim][n])
    cfmm::DevBuf<double> xr, xi, nr, ni;
    cfmm::DevBuf<uint64_t> keys;
    cfmm::DevBuf<int> perm;
    cfmm::TreeDev tree;
    std::vector<int> P;              // per level
    // expansions: per box coefficient offsets (in complex units), levels >= l0
    std::vector<int64_t> exp_off_h;
    cfmm::DevBuf<int64_t> exp_off;
    cfmm::DevBuf<int> box_P;         // P of the box's level
    int64_t ncoef = 0;               // complex coefficients per rhs per kind
    int maxP = 0;
    // workspaces (grown on demand)
    cfmm::DevBuf<cd> mpole, local, dens_s, out_s, m2l_part;
    cfmm::DevBuf<cd> grad_s;         // sorted target gradient [nrhs][dim][n] (cfmm_apply_grad)
    int grad_nrhs = 0;
    cfmm::DevBuf<double> staging;
    int ws_nrhs = 0;
    // diagnostics
    int64_t p2p_pairs = 0, m2l_pairs = 0;
    bool timing = false;
    bool serial = false;             // timing mode 2: the near field on the plan's stream
    double step_ms[9] = {0};
    cudaEvent_t ev[10] = {};
    // near field (List 1) on a second stream, concurrent with the far field:
    // fork after the permuted densities, join before the expansions are
    // evaluated into the same output
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_p2p[2] = {};
    bool p2p_side = false;           // the last apply ran the near field on `side`
    bool p2p_serial = false;         // the last apply ran it in line (timing mode 2)
    // captured apply
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_kernels = 0;       // kernel nodes recorded in `graph`
};
