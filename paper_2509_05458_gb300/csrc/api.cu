// The C ABI (include/cfmm.h): argument checking, host/device staging, plan
// life cycle, error reporting, and the host-side tables (Gauss-Laguerre rule
// by Golub-Welsch).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>

#include "cfmm_special.cuh"
#include "kernels.cuh"

namespace cfmm {

static thread_local int g_status = 0;
static thread_local std::string g_msg;

void set_error(int status, const std::string& msg) {
    g_status = status;
    g_msg = msg;
}

std::atomic<int64_t>& launch_counter() {
    static std::atomic<int64_t> c{0};
    return c;
}

// failure injection (tests): the next g_fail_allocs device allocations fail
static std::atomic<int> g_fail_allocs{0};
static void injected_failure() {
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1))
            throw Error{CFMM_ENOMEM, "device allocation failed (injected)"};
    }
}

void* Scratch::take(size_t bytes) {
    injected_failure();
    bytes = (bytes + 255) & ~(size_t)255;
    while (cur_ < chunks_.size()) {
        if (off_ + bytes <= chunks_[cur_].size) {
            void* p = chunks_[cur_].p + off_;
            off_ += bytes;
            return p;
        }
        ++cur_;
        off_ = 0;
    }
    size_t sz = std::max(bytes, (size_t)64 << 20);
    char* p = nullptr;
    CFMM_CUDA(cudaMalloc((void**)&p, sz));
    chunks_.push_back(Chunk{p, sz});
    cur_ = chunks_.size() - 1;
    off_ = bytes;
    return p;
}

// ---- caching device allocator -------------------------------------------
// Size classes: powers of two from 256 B to 64 MiB, then multiples of 64 MiB.
// At most kPoolCap bytes are kept per device; beyond that freed blocks go back
// to the driver. An allocation that fails releases the device's cache and is
// retried once.
namespace {
constexpr size_t kPoolCap = (size_t)8 << 30;
struct PoolDev {
    std::map<size_t, std::vector<void*>> free;
    size_t cached = 0;
};
std::mutex g_pool_mu;
std::map<int, PoolDev>& pool_devs() {
    static std::map<int, PoolDev> m;
    return m;
}
size_t pool_class(size_t b) {
    const size_t big = (size_t)64 << 20;
    if (b > big) return (b + big - 1) / big * big;
    size_t s = 256;
    while (s < b) s <<= 1;
    return s;
}
}  // namespace

void* pool_alloc(size_t bytes, int* dev_out) {
    injected_failure();
    int dev = 0;
    CFMM_CUDA(cudaGetDevice(&dev));
    *dev_out = dev;
    size_t sz = pool_class(bytes);
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        PoolDev& D = pool_devs()[dev];
        auto it = D.free.find(sz);
        if (it != D.free.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            D.cached -= sz;
            return p;
        }
    }
    void* p = nullptr;
    if (cudaMalloc(&p, sz) != cudaSuccess) {
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(g_pool_mu);
            PoolDev& D = pool_devs()[dev];
            cudaDeviceSynchronize();
            for (auto& kv : D.free)
                for (void* q : kv.second) cudaFree(q);
            D.free.clear();
            D.cached = 0;
        }
        if (cudaMalloc(&p, sz) != cudaSuccess) {
            cudaGetLastError();
            throw Error{CFMM_ENOMEM, "device allocation failed"};
        }
    }
    return p;
}

void pool_free(void* p, size_t bytes, int dev) {
    if (!p) return;
    size_t sz = pool_class(bytes);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    PoolDev& D = pool_devs()[dev];
    if (D.cached + sz > kPoolCap) {
        cudaFree(p);
        return;
    }
    D.free[sz].push_back(p);
    D.cached += sz;
}

Scratch::~Scratch() {
    for (auto& c : chunks_) cudaFree(c.p);
}

void* HostStage::take(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    while (cur_ < chunks_.size()) {
        if (off_ + bytes <= chunks_[cur_].size) {
            void* p = chunks_[cur_].p + off_;
            off_ += bytes;
            return p;
        }
        ++cur_;
        off_ = 0;
    }
    size_t sz = std::max(bytes, (size_t)4 << 20);
    char* p = nullptr;
    CFMM_CUDA(cudaHostAlloc((void**)&p, sz, cudaHostAllocDefault));
    chunks_.push_back(Chunk{p, sz});
    cur_ = chunks_.size() - 1;
    off_ = bytes;
    return p;
}

HostStage::~HostStage() {
    for (auto& c : chunks_) cudaFreeHost(c.p);
}

HostStage& plan_host_stage() {
    thread_local HostStage stage;
    return stage;
}

void upload(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return;
    void* h = plan_host_stage().take(bytes);
    std::memcpy(h, src, bytes);
    CFMM_CUDA(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, st));
}

Scratch& plan_scratch() {
    thread_local std::vector<std::unique_ptr<Scratch>> per_dev;
    int dev = 0;
    CFMM_CUDA(cudaGetDevice(&dev));
    if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1);
    if (!per_dev[dev]) per_dev[dev].reset(new Scratch());
    return *per_dev[dev];
}

// ---- Gauss-Laguerre rules (generalized, alpha = -1/2 and +1/2) ----------
// Golub-Welsch: the nodes are the eigenvalues of the symmetric tridiagonal
// Jacobi matrix of the monic Laguerre recurrence (diagonal 2i+alpha+1,
// off-diagonal sqrt(i (i+alpha))), the weights Gamma(alpha+1) times the
// squared first components of the normalised eigenvectors. The eigenproblem
// is solved by implicit QL iterations with Wilkinson shifts, tracking only the
// first row of the eigenvector matrix.
static void gauss_laguerre(double alpha, int n, double* x, double* w) {
    std::vector<double> d(n), e(n, 0.0), z(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = 2.0 * i + alpha + 1.0;
    for (int i = 1; i < n; ++i) e[i - 1] = std::sqrt(i * (i + alpha));
    z[0] = 1.0;
    for (int l = 0; l < n; ++l) {
        for (int iter = 0; iter < 200; ++iter) {
            int m = l;
            for (; m < n - 1; ++m) {
                double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-17 * dd) break;
            }
            if (m == l) break;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            for (; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                double zf = z[i + 1];
                z[i + 1] = s * z[i] + c * zf;
                z[i] = c * z[i] - s * zf;
            }
            if (r == 0.0 && i >= l) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
    double g0 = std::tgamma(alpha + 1.0);
    for (int i = 0; i < n; ++i) {
        x[i] = d[idx[i]];
        w[i] = g0 * z[idx[i]] * z[idx[i]];
    }
}

const LagRule& host_lag_rule() {
    static LagRule R;
    static std::once_flag once;
    std::call_once(once, [] {
        gauss_laguerre(-0.5, kLagNodes, R.x[0], R.w[0]);
        gauss_laguerre(0.5, kLagNodes, R.x[1], R.w[1]);
    });
    return R;
}

void ensure_device_tables() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    CFMM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)done.size() <= dev) done.resize(dev + 1, 0);
    if (done[dev]) return;
    host_lag_rule();
    upload_lag_rule_p2p();
    upload_lag_rule_fmm2d();
    done[dev] = 1;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// a device view of a caller array (host or device) of `count` doubles: device
// pointers are used in place, host arrays are copied into plan scratch
static const double* stage_in(const double* src, size_t count, cudaStream_t st) {
    if (is_device_ptr(src)) return src;
    double* dst = plan_scratch().take_n<double>(count);
    CFMM_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyHostToDevice, st));
    return dst;
}

template <class F>
static int guarded(F f) {
    try {
        f();
        return 0;
    } catch (const Error& e) {
        set_error(e.status, e.msg);
        return e.status;
    } catch (const std::exception& e) {
        set_error(CFMM_ECUDA, e.what());
        return CFMM_ECUDA;
    }
}

// ---- apply-path helpers (permutation of densities and results) -----------
// densities [nrhs][ncomp][nsrc] in the caller's order -> sorted [nrhs][n];
// union points beyond the sources (separate targets) carry zero density
__global__ void k_permute_dens(const cd* __restrict__ dens, const int* __restrict__ perm, int64_t n, int64_t nsrc,
                               int nrhs, int ncomp, int comp, cd* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (i >= n) return;
    int64_t j = perm[i];
    out[(int64_t)r * n + i] = j < nsrc ? dens[((int64_t)r * ncomp + comp) * nsrc + j] : cd{0.0, 0.0};
}

// sorted [nrhs][n] -> the caller's [nrhs][nout] at union indices [first, first + nout)
__global__ void k_unpermute(const cd* __restrict__ us, const int* __restrict__ perm, int64_t n, int64_t first,
                            int64_t nout, cd scale, cd* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (i >= n) return;
    int64_t j = (int64_t)perm[i] - first;
    if (j < 0 || j >= nout) return;
    cd v = us[(int64_t)r * n + i];
    out[(int64_t)r * nout + j] = v * scale;
}

static void record(cfmm_plan_s* P, int i) {
    if (P->timing) CFMM_CUDA(cudaEventRecord(P->ev[i], P->stream));
}

cudaStream_t near_fork(cfmm_plan_s* P) {
    if (P->timing && P->serial) {
        CFMM_CUDA(cudaEventRecord(P->ev_p2p[0], P->stream));
        P->p2p_serial = true;
        return P->stream;
    }
    CFMM_CUDA(cudaEventRecord(P->ev_fork, P->stream));
    CFMM_CUDA(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
    if (P->timing) CFMM_CUDA(cudaEventRecord(P->ev_p2p[0], P->side));
    P->p2p_side = true;
    return P->side;
}

void near_launched(cfmm_plan_s* P) {
    if (P->p2p_serial) CFMM_CUDA(cudaEventRecord(P->ev_p2p[1], P->stream));
}

void near_join(cfmm_plan_s* P) {
    if (P->p2p_serial) return;
    if (P->timing) CFMM_CUDA(cudaEventRecord(P->ev_p2p[1], P->side));
    CFMM_CUDA(cudaEventRecord(P->ev_join, P->side));
    CFMM_CUDA(cudaStreamWaitEvent(P->stream, P->ev_join, 0));
}

// the full apply on device buffers (densities [nrhs][ncomp][n], out [nrhs][n])
static void apply_device(cfmm_plan_s* P, const cd* dens, int nrhs, cd* out, cd* grad = nullptr) {
    cudaStream_t st = P->stream;
    int64_t n = P->n;
    int ncomp = (P->slp ? 1 : 0) + (P->dlp ? 1 : 0);
    if (P->ws_nrhs < nrhs) {
        P->dens_s.alloc((size_t)n * nrhs * ncomp);
        P->out_s.alloc((size_t)n * nrhs);
        P->ws_nrhs = nrhs;
    }
    cd* gs = nullptr;
    if (grad) {
        if (P->grad_nrhs < nrhs) {
            P->grad_s.alloc((size_t)n * nrhs * P->dim);
            P->grad_nrhs = nrhs;
        }
        gs = P->grad_s.get();
    }
    cd* sg = P->slp ? P->dens_s.get() : nullptr;
    cd* ta = P->dlp ? P->dens_s.get() + (P->slp ? (int64_t)n * nrhs : 0) : nullptr;
    P->p2p_side = false;
    P->p2p_serial = false;
    record(P, 0);
    dim3 g((unsigned)((n + 255) / 256), nrhs);
    int comp = 0;
    if (P->slp) {
        k_permute_dens<<<g, 256, 0, st>>>(dens, P->perm.get(), n, P->n_src, nrhs, ncomp, comp++, sg);
        CFMM_LAUNCHED();
    }
    if (P->dlp) {
        k_permute_dens<<<g, 256, 0, st>>>(dens, P->perm.get(), n, P->n_src, nrhs, ncomp, comp++, ta);
        CFMM_LAUNCHED();
    }
    record(P, 1);
    if (P->dim == 2) fmm2d_apply(P, sg, ta, n, P->out_s.get(), nrhs, gs);
    else if (P->kernel == CFMM_HELMHOLTZ) helm3d_apply(P, sg, ta, n, P->out_s.get(), nrhs, gs);
    else fmm3d_apply(P, sg, ta, n, P->out_s.get(), nrhs, gs);
    record(P, 8);
    cd scale = P->green ? green_scale(P->dim, P->kernel) : cd{1.0, 0.0};
    int64_t first = P->n_trg > 0 ? P->n_src : 0, nout = P->n_trg > 0 ? P->n_trg : n;
    if (out) {
        k_unpermute<<<g, 256, 0, st>>>(P->out_s.get(), P->perm.get(), n, first, nout, scale, out);
        CFMM_LAUNCHED();
    }
    if (grad) {
        // the gradient's dim components are rows of their own
        dim3 gg((unsigned)((n + 255) / 256), nrhs * P->dim);
        k_unpermute<<<gg, 256, 0, st>>>(gs, P->perm.get(), n, first, nout, scale, grad);
        CFMM_LAUNCHED();
    }
    record(P, 9);
    if (P->timing) {
        CFMM_CUDA(cudaEventSynchronize(P->ev[9]));
        for (int i = 0; i < 9; ++i) {
            float ms = 0.f;
            CFMM_CUDA(cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]));
            P->step_ms[i] = ms;
        }
        if (P->p2p_side || P->p2p_serial) {
            // the near field's own duration (beside the far field, or in line)
            float ms = 0.f;
            CFMM_CUDA(cudaEventElapsedTime(&ms, P->ev_p2p[0], P->ev_p2p[1]));
            P->step_ms[6] = ms;
            // in line it is launched inside the P2M bracket
            if (P->p2p_serial) P->step_ms[1] -= ms;
        }
    }
}

static void destroy_plan(cfmm_plan_s* P) {
    if (!P) return;
    // queued work of this plan must finish before its buffers return to the pool
    cudaStreamSynchronize(P->stream);
    if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    fmm2d_release(P);
    fmm3d_release(P);
    helm3d_release(P);
    for (auto& e : P->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : P->ev_p2p)
        if (e) cudaEventDestroy(e);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    if (P->side) {
        cudaStreamSynchronize(P->side);
        cudaStreamDestroy(P->side);
    }
    delete P;
}

}  // namespace cfmm

// One CUDA graph over the applies of several plans (a batch of geometries).
struct cfmm_batch_s {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;              // kernel nodes in the graph
    std::vector<cudaEvent_t> ev;      // fork + one join per member
};

namespace cfmm {
static void destroy_batch(cfmm_batch_s* B) {
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (auto& e : B->ev)
        if (e) cudaEventDestroy(e);
    delete B;
}
}  // namespace cfmm

using namespace cfmm;

extern "C" {

int cfmm_last_status(void) { return g_status; }
const char* cfmm_last_error(void) { return g_msg.c_str(); }
const char* cfmm_version(void) { return "cfmm-gb300 0.1 (sm_103a)"; }
int64_t cfmm_launch_count(void) { return launch_counter().load(); }

int cfmm_debug_fail_allocs(int count) {
    return guarded([&] {
        CFMM_REQUIRE(count >= 0, CFMM_EINVAL, "count must be >= 0");
        g_fail_allocs.store(count);
    });
}

// cfmm_plan_ex and cfmm_plan_targets: sources [0, m) and (when n > 0) separate
// targets [m, m + n) of the tree's points
static cfmm_plan_t plan_common(int dim, int kernel, double k, double eps, const double* src_re,
                               const double* src_im, const double* nrm_re, const double* nrm_im, int64_t m,
                               const double* trg_re, const double* trg_im, int64_t ntrg, const cfmm_opts* opts) {
    cfmm_plan_s* P = nullptr;
    int rc = guarded([&] {
        CFMM_REQUIRE(dim == 2 || dim == 3, CFMM_EINVAL, "dim must be 2 or 3");
        int ker = kernel & 0xF;
        CFMM_REQUIRE(ker == CFMM_LAPLACE || ker == CFMM_HELMHOLTZ, CFMM_EINVAL, "kernel must be LAPLACE or HELMHOLTZ");
        CFMM_REQUIRE((kernel & ~(0xF | CFMM_SLP | CFMM_DLP | CFMM_GREEN_SCALE)) == 0, CFMM_EINVAL, "unknown kernel flags");
        CFMM_REQUIRE(ker == CFMM_LAPLACE || (std::isfinite(k) && k > 0.0), CFMM_EINVAL, "Helmholtz needs k > 0");
        CFMM_REQUIRE(std::isfinite(eps) && eps >= 1e-15 && eps <= 0.1, CFMM_EINVAL, "eps must be in [1e-15, 0.1]");
        CFMM_REQUIRE(m >= 1 && ntrg >= 0 && m + ntrg < ((int64_t)1 << 31), CFMM_EINVAL,
                     "point counts must be >= 1 (sources), >= 0 (targets), below 2^31 in total");
        CFMM_REQUIRE(src_re && src_im, CFMM_EINVAL, "points are required");
        CFMM_REQUIRE(ntrg == 0 || (trg_re && trg_im), CFMM_EINVAL, "target points are required");
        bool dlp = (kernel & CFMM_DLP) != 0;
        bool slp = (kernel & CFMM_SLP) != 0 || !dlp;
        CFMM_REQUIRE(!dlp || (nrm_re && nrm_im), CFMM_EINVAL, "double layer needs normals");
        cfmm_opts o{};
        if (opts) o = *opts;
        int leaf = o.leaf_size > 0 ? o.leaf_size : 64;
        // sep: 0 = default 1, < 0 = automatic (chosen in build_tree from the
        // Lipschitz estimate)
        int sep = o.sep > 0 ? o.sep : o.sep < 0 ? 0 : 1;
        CFMM_REQUIRE(leaf <= 4096, CFMM_EINVAL, "leaf_size must be <= 4096");
        CFMM_REQUIRE(sep <= 3, CFMM_EINVAL, "sep must be 1, 2 or 3 (or < 0 for automatic)");
        CFMM_REQUIRE(o.precision >= 0 && o.precision <= 2, CFMM_EINVAL, "bad precision mode");
        CFMM_REQUIRE(o.top_level >= CFMM_TOP_FIT, CFMM_EINVAL, "top_level must be >= -1 (CFMM_TOP_FIT)");
        int64_t n = m + ntrg;
        P = new cfmm_plan_s();
        P->dim = dim;
        P->kernel = ker;
        P->flags = kernel;
        P->slp = slp;
        P->dlp = dlp;
        P->green = (kernel & CFMM_GREEN_SCALE) != 0;
        P->kappa = ker == CFMM_HELMHOLTZ ? k : 0.0;
        P->eps = eps;
        P->n = n;
        P->n_src = m;
        P->n_trg = ntrg;
        P->leaf_size = leaf;
        P->sep = sep;
        P->precision = o.precision == CFMM_AUTO ? (eps >= 1e-5 ? CFMM_MIXED : CFMM_FP64) : o.precision;
        P->stream = (cudaStream_t)o.stream;
        CFMM_CUDA(cudaGetDevice(&P->device));
        ensure_device_tables();
        for (auto& e : P->ev) CFMM_CUDA(cudaEventCreate(&e));
        for (auto& e : P->ev_p2p) CFMM_CUDA(cudaEventCreate(&e));
        CFMM_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
        CFMM_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
        CFMM_CUDA(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
        Scratch& scr = plan_scratch();
        scr.rewind();
        plan_host_stage().rewind();
        size_t cs = (size_t)m * dim, ct = (size_t)ntrg * dim;
        const double *re, *im, *nre = nullptr, *nim = nullptr;
        if (ntrg == 0) {
            re = stage_in(src_re, cs, P->stream);
            im = stage_in(src_im, cs, P->stream);
            nre = dlp ? stage_in(nrm_re, cs, P->stream) : nullptr;
            nim = dlp ? stage_in(nrm_im, cs, P->stream) : nullptr;
        } else {
            // the tree's points: sources then targets (targets get zero normals)
            auto cat = [&](const double* a, const double* b) {
                double* d = scr.take_n<double>(cs + ct);
                CFMM_CUDA(cudaMemcpyAsync(d, a, cs * sizeof(double), cudaMemcpyDefault, P->stream));
                if (b) CFMM_CUDA(cudaMemcpyAsync(d + cs, b, ct * sizeof(double), cudaMemcpyDefault, P->stream));
                else CFMM_CUDA(cudaMemsetAsync(d + cs, 0, ct * sizeof(double), P->stream));
                return (const double*)d;
            };
            re = cat(src_re, trg_re);
            im = cat(src_im, trg_im);
            if (dlp) {
                nre = cat(nrm_re, nullptr);
                nim = cat(nrm_im, nullptr);
            }
        }
        build_tree(P, re, im, nre, nim, o.top_level);
        if (dim == 2) fmm2d_presetup(P);   // its row table overlaps the lists
        build_plan_lists(P);
        if (dim == 2) fmm2d_setup(P);
        else if (P->kernel == CFMM_HELMHOLTZ) helm3d_setup(P);
        else fmm3d_setup(P);
        CFMM_CUDA(cudaStreamSynchronize(P->stream));
        scr.rewind();
        plan_host_stage().rewind();
    });
    if (rc != 0) {
        destroy_plan(P);
        return nullptr;
    }
    return P;
}

cfmm_plan_t cfmm_plan_ex(int dim, int kernel, double k, double eps, const double* pts_re, const double* pts_im,
                         const double* nrm_re, const double* nrm_im, int64_t n, const cfmm_opts* opts) {
    if (n < 1) {
        guarded([&] { CFMM_REQUIRE(false, CFMM_EINVAL, "n must be in [1, 2^31)"); });
        return nullptr;
    }
    return plan_common(dim, kernel, k, eps, pts_re, pts_im, nrm_re, nrm_im, n, nullptr, nullptr, 0, opts);
}

cfmm_plan_t cfmm_plan_targets(int dim, int kernel, double k, double eps, const double* src_re, const double* src_im,
                              const double* nrm_re, const double* nrm_im, int64_t m, const double* trg_re,
                              const double* trg_im, int64_t n, const cfmm_opts* opts) {
    if (n < 1) {
        guarded([&] { CFMM_REQUIRE(false, CFMM_EINVAL, "the target count must be >= 1"); });
        return nullptr;
    }
    return plan_common(dim, kernel, k, eps, src_re, src_im, nrm_re, nrm_im, m, trg_re, trg_im, n, opts);
}

cfmm_plan_t cfmm_plan(int dim, int kernel, double k, double eps, const double* pts_re, const double* pts_im,
                      int64_t n) {
    return cfmm_plan_ex(dim, kernel, k, eps, pts_re, pts_im, nullptr, nullptr, n, nullptr);
}

int cfmm_apply(cfmm_plan_t P, const double* densities, int nrhs, double* out) {
    return guarded([&] {
        CFMM_REQUIRE(P, CFMM_EINVAL, "null plan");
        CFMM_REQUIRE(nrhs >= 1, CFMM_EINVAL, "nrhs must be >= 1");
        CFMM_REQUIRE(densities && out, CFMM_EINVAL, "densities and out are required");
        int ncomp = (P->slp ? 1 : 0) + (P->dlp ? 1 : 0);
        int64_t nout = P->n_trg > 0 ? P->n_trg : P->n;
        size_t din = (size_t)nrhs * ncomp * P->n_src * 2, dout = (size_t)nrhs * nout * 2;
        bool dev_in = is_device_ptr(densities), dev_out = is_device_ptr(out);
        const cd* d_in = reinterpret_cast<const cd*>(densities);
        cd* d_out = reinterpret_cast<cd*>(out);
        DevBuf<double> sin_, sout;
        if (!dev_in) {
            P->staging.alloc(din + dout);
            CFMM_CUDA(cudaMemcpyAsync(P->staging.get(), densities, din * sizeof(double), cudaMemcpyHostToDevice,
                                      P->stream));
            d_in = reinterpret_cast<const cd*>(P->staging.get());
        }
        if (!dev_out) {
            P->staging.alloc(din + dout);
            d_out = reinterpret_cast<cd*>(P->staging.get() + din);
            if (!dev_in) d_in = reinterpret_cast<const cd*>(P->staging.get());
        }
        apply_device(P, d_in, nrhs, d_out);
        if (!dev_out) {
            CFMM_CUDA(cudaMemcpyAsync(out, d_out, dout * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
            CFMM_CUDA(cudaStreamSynchronize(P->stream));
        }
    });
}

int cfmm_apply_grad(cfmm_plan_t P, const double* densities, int nrhs, double* out, double* grad) {
    return guarded([&] {
        CFMM_REQUIRE(P, CFMM_EINVAL, "null plan");
        CFMM_REQUIRE(nrhs >= 1, CFMM_EINVAL, "nrhs must be >= 1");
        CFMM_REQUIRE(densities && grad, CFMM_EINVAL, "densities and grad are required");
        int ncomp = (P->slp ? 1 : 0) + (P->dlp ? 1 : 0);
        int64_t nout = P->n_trg > 0 ? P->n_trg : P->n;
        size_t din = (size_t)nrhs * ncomp * P->n_src * 2, dout = out ? (size_t)nrhs * nout * 2 : 0,
               dgrad = (size_t)nrhs * P->dim * nout * 2;
        bool dev_in = is_device_ptr(densities), dev_out = !out || is_device_ptr(out), dev_g = is_device_ptr(grad);
        const cd* d_in = reinterpret_cast<const cd*>(densities);
        cd* d_out = reinterpret_cast<cd*>(out);
        cd* d_g = reinterpret_cast<cd*>(grad);
        if (!dev_in || !dev_out || !dev_g) {
            P->staging.alloc(din + dout + dgrad);
            double* base = P->staging.get();
            if (!dev_in) {
                CFMM_CUDA(cudaMemcpyAsync(base, densities, din * sizeof(double), cudaMemcpyHostToDevice, P->stream));
                d_in = reinterpret_cast<const cd*>(base);
            }
            if (!dev_out) d_out = reinterpret_cast<cd*>(base + din);
            if (!dev_g) d_g = reinterpret_cast<cd*>(base + din + dout);
        }
        apply_device(P, d_in, nrhs, d_out, d_g);
        if (!dev_out) CFMM_CUDA(cudaMemcpyAsync(out, d_out, dout * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
        if (!dev_g) CFMM_CUDA(cudaMemcpyAsync(grad, d_g, dgrad * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
        if (!dev_out || !dev_g) CFMM_CUDA(cudaStreamSynchronize(P->stream));
    });
}

int cfmm_apply_capture(cfmm_plan_t P, const double* densities, int nrhs, double* out) {
    return guarded([&] {
        CFMM_REQUIRE(P, CFMM_EINVAL, "null plan");
        CFMM_REQUIRE(P->stream != nullptr, CFMM_EINVAL, "capture needs a plan created on a non-NULL stream");
        CFMM_REQUIRE(nrhs >= 1 && densities && out, CFMM_EINVAL, "bad arguments");
        CFMM_REQUIRE(is_device_ptr(densities) && is_device_ptr(out), CFMM_EINVAL, "capture takes device pointers");
        const cd* d_in = reinterpret_cast<const cd*>(densities);
        cd* d_out = reinterpret_cast<cd*>(out);
        bool timing = P->timing;
        P->timing = false;
        // one eager apply sizes every workspace, so nothing is allocated while capturing
        apply_device(P, d_in, nrhs, d_out);
        CFMM_CUDA(cudaStreamSynchronize(P->stream));
        if (P->graph_exec) {
            cudaGraphExecDestroy(P->graph_exec);
            P->graph_exec = nullptr;
        }
        if (P->graph) {
            cudaGraphDestroy(P->graph);
            P->graph = nullptr;
        }
        int64_t c0 = launch_counter().load();
        CFMM_CUDA(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
        try {
            apply_device(P, d_in, nrhs, d_out);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(P->stream, &g);
            if (g) cudaGraphDestroy(g);
            P->timing = timing;
            throw;
        }
        // the kernels were recorded, not launched: count them at each replay
        P->graph_kernels = launch_counter().load() - c0;
        launch_counter().fetch_sub(P->graph_kernels);
        CFMM_CUDA(cudaStreamEndCapture(P->stream, &P->graph));
        CFMM_CUDA(cudaGraphInstantiate(&P->graph_exec, P->graph, 0));
        P->timing = timing;
    });
}

int cfmm_apply_replay(cfmm_plan_t P) {
    return guarded([&] {
        CFMM_REQUIRE(P && P->graph_exec, CFMM_EINVAL, "no captured apply");
        CFMM_CUDA(cudaGraphLaunch(P->graph_exec, P->stream));
        count_launch((int)P->graph_kernels);
    });
}

cfmm_batch_t cfmm_batch_capture(const cfmm_plan_t* plans, int count, const double* const* densities,
                                const int* nrhs, double* const* out, void* stream) {
    auto* B = new cfmm_batch_s;
    std::vector<std::pair<cfmm_plan_s*, bool>> saved;
    int rc = guarded([&] {
        CFMM_REQUIRE(plans && densities && nrhs && out && count >= 1, CFMM_EINVAL, "bad arguments");
        CFMM_REQUIRE(stream != nullptr, CFMM_EINVAL, "batch capture needs a non-NULL stream");
        B->stream = (cudaStream_t)stream;
        int dev = 0;
        CFMM_CUDA(cudaGetDevice(&dev));
        for (int i = 0; i < count; ++i) {
            cfmm_plan_s* P = plans[i];
            CFMM_REQUIRE(P, CFMM_EINVAL, "null plan in batch");
            CFMM_REQUIRE(P->stream != nullptr, CFMM_EINVAL, "every plan of a batch needs a non-NULL stream");
            CFMM_REQUIRE(P->device == dev, CFMM_EINVAL, "every plan of a batch must live on the current device");
            CFMM_REQUIRE(nrhs[i] >= 1 && densities[i] && out[i], CFMM_EINVAL, "bad batch member arguments");
            CFMM_REQUIRE(is_device_ptr(densities[i]) && is_device_ptr(out[i]), CFMM_EINVAL,
                         "batch capture takes device pointers");
        }
        for (int i = 0; i < count; ++i) {
            saved.push_back({plans[i], plans[i]->timing});
            plans[i]->timing = false;
        }
        auto din = [&](int i) { return reinterpret_cast<const cd*>(densities[i]); };
        auto dout = [&](int i) { return reinterpret_cast<cd*>(out[i]); };
        // one eager apply per member sizes every workspace, so nothing is
        // allocated while capturing
        for (int i = 0; i < count; ++i) apply_device(plans[i], din(i), nrhs[i], dout(i));
        for (int i = 0; i < count; ++i) CFMM_CUDA(cudaStreamSynchronize(plans[i]->stream));
        B->ev.assign(count + 1, nullptr);
        for (auto& e : B->ev) CFMM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        int64_t c0 = launch_counter().load();
        CFMM_CUDA(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
        try {
            // fork: every member stream waits for the batch stream, runs its
            // apply, and the batch stream joins them all
            CFMM_CUDA(cudaEventRecord(B->ev[0], B->stream));
            for (int i = 0; i < count; ++i) {
                cudaStream_t ps = plans[i]->stream;
                if (ps != B->stream) CFMM_CUDA(cudaStreamWaitEvent(ps, B->ev[0], 0));
                apply_device(plans[i], din(i), nrhs[i], dout(i));
                if (ps != B->stream) {
                    CFMM_CUDA(cudaEventRecord(B->ev[i + 1], ps));
                    CFMM_CUDA(cudaStreamWaitEvent(B->stream, B->ev[i + 1], 0));
                }
            }
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(B->stream, &g);
            if (g) cudaGraphDestroy(g);
            launch_counter().store(c0);
            throw;
        }
        B->kernels = launch_counter().load() - c0;
        launch_counter().fetch_sub(B->kernels);
        CFMM_CUDA(cudaStreamEndCapture(B->stream, &B->graph));
        CFMM_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
    });
    for (auto& s : saved) s.first->timing = s.second;
    if (rc != 0) {
        destroy_batch(B);
        return nullptr;
    }
    return B;
}

int cfmm_batch_replay(cfmm_batch_t B) {
    return guarded([&] {
        CFMM_REQUIRE(B && B->exec, CFMM_EINVAL, "no captured batch");
        CFMM_CUDA(cudaGraphLaunch(B->exec, B->stream));
        count_launch((int)B->kernels);
    });
}

int64_t cfmm_batch_kernels(cfmm_batch_t B) { return B ? B->kernels : 0; }

int cfmm_batch_destroy(cfmm_batch_t B) {
    return guarded([&] { destroy_batch(B); });
}

int cfmm_destroy(cfmm_plan_t P) {
    return guarded([&] { destroy_plan(P); });
}

int cfmm_direct(int dim, int kernel, double k, const double* src_re, const double* src_im, const double* nrm_re,
                const double* nrm_im, int64_t m, const double* trg_re, const double* trg_im, int64_t n,
                const double* densities, int nrhs, double* out, int precision, void* stream) {
    return guarded([&] {
        CFMM_REQUIRE(dim == 2 || dim == 3, CFMM_EINVAL, "dim must be 2 or 3");
        int ker = kernel & 0xF;
        CFMM_REQUIRE(ker == CFMM_LAPLACE || ker == CFMM_HELMHOLTZ, CFMM_EINVAL, "bad kernel");
        CFMM_REQUIRE(ker == CFMM_LAPLACE || (std::isfinite(k) && k > 0.0), CFMM_EINVAL, "Helmholtz needs k > 0");
        CFMM_REQUIRE(m >= 1 && n >= 1 && nrhs >= 1, CFMM_EINVAL, "sizes must be positive");
        CFMM_REQUIRE(precision == CFMM_FP64 || precision == CFMM_MIXED, CFMM_EINVAL,
                     "direct sum: precision must be CFMM_FP64 or CFMM_MIXED");
        bool dlp = (kernel & CFMM_DLP) != 0;
        bool slp = (kernel & CFMM_SLP) != 0 || !dlp;
        CFMM_REQUIRE(!dlp || (nrm_re && nrm_im), CFMM_EINVAL, "double layer needs normals");
        CFMM_REQUIRE(is_device_ptr(src_re) && is_device_ptr(trg_re) && is_device_ptr(densities) &&
                         is_device_ptr(out),
                     CFMM_EINVAL, "cfmm_direct takes device pointers");
        ensure_device_tables();
        cudaStream_t st = (cudaStream_t)stream;
        // SoA copies of the [n][dim] inputs
        auto soa = [&](DevBuf<double>& dst, const double* src, int64_t cnt) {
            std::vector<double> tmp;
            dst.alloc((size_t)cnt * dim);
            // transpose on device through a small kernel-free path: 2D copy
            CFMM_CUDA(cudaMemcpy2DAsync(dst.get(), sizeof(double), src, dim * sizeof(double), sizeof(double), cnt,
                                        cudaMemcpyDeviceToDevice, st));
            for (int a = 1; a < dim; ++a)
                CFMM_CUDA(cudaMemcpy2DAsync(dst.get() + a * cnt, sizeof(double), src + a, dim * sizeof(double),
                                            sizeof(double), cnt, cudaMemcpyDeviceToDevice, st));
        };
        DevBuf<double> sr, si, nr, ni, tr, ti;
        soa(sr, src_re, m);
        soa(si, src_im, m);
        soa(tr, trg_re, n);
        soa(ti, trg_im, n);
        if (dlp) {
            soa(nr, nrm_re, m);
            soa(ni, nrm_im, m);
        }
        int ncomp = (slp ? 1 : 0) + (dlp ? 1 : 0);
        // densities [nrhs][ncomp][m]: sigma = comp 0, tau = last comp; stride between rhs = ncomp*m
        const cd* d = reinterpret_cast<const cd*>(densities);
        KParams K{sr.get(), si.get(), dlp ? nr.get() : nullptr, dlp ? ni.get() : nullptr, tr.get(), ti.get(), m, n,
                  slp ? d : nullptr, dlp ? d + (slp ? m : 0) : nullptr, ncomp * m, slp, dlp, k};
        launch_direct(dim, ker, K, reinterpret_cast<cd*>(out), nrhs, st, precision == CFMM_MIXED);
        if (kernel & CFMM_GREEN_SCALE) launch_scale_inplace(reinterpret_cast<cd*>(out), n * nrhs, green_scale(dim, ker), st);
        CFMM_CUDA(cudaStreamSynchronize(st));
    });
}

int cfmm_direct_noalloc(int dim, int kernel, double k, const double* src_re, const double* src_im,
                        const double* nrm_re, const double* nrm_im, int64_t m, const double* trg_re,
                        const double* trg_im, int64_t n, const double* densities, int nrhs, double* out,
                        void* stream) {
    return guarded([&] {
        direct_noalloc(dim, kernel, k, src_re, src_im, nrm_re, nrm_im, m, trg_re, trg_im, n, densities, nrhs, out,
                       stream);
    });
}

int cfmm_plan_get_info(cfmm_plan_t P, cfmm_plan_info* info) {
    return guarded([&] {
        CFMM_REQUIRE(P && info, CFMM_EINVAL, "null argument");
        memset(info, 0, sizeof(*info));
        info->dim = P->dim;
        info->kernel = P->flags;
        info->sep = P->sep;
        info->leaf_size = P->leaf_size;
        info->precision = P->precision;
        info->nlevels = P->tree.nlevels;
        info->nboxes = P->tree.nboxes;
        info->nleaves = P->tree.nleaves;
        info->l0 = P->tree.l0;
        info->n = P->n;
        info->n_src = P->n_src;
        info->n_trg = P->n_trg;
        for (int w = 0; w < 4; ++w) info->list_len[w] = P->tree.llen[w];
        info->p2p_pairs = P->p2p_pairs;
        info->m2l_pairs = P->m2l_pairs;
        for (int d = 0; d < 3; ++d) info->root_lo[d] = P->lo[d];
        info->root_width = P->W;
        info->lipschitz = P->lipschitz;
    });
}

int cfmm_plan_get_orders(cfmm_plan_t P, int* p, int nlevels) {
    return guarded([&] {
        CFMM_REQUIRE(P && p, CFMM_EINVAL, "null argument");
        for (int i = 0; i < nlevels && i < (int)P->P.size(); ++i) p[i] = P->P[i];
    });
}

int cfmm_plan_export_tree(cfmm_plan_t P, int64_t* perm, uint64_t* keys, int32_t* box_level, uint64_t* box_prefix,
                          int32_t* box_start, int32_t* box_end, int32_t* box_leaf, int32_t* box_parent,
                          double* center_re, double* center_im) {
    return guarded([&] {
        CFMM_REQUIRE(P, CFMM_EINVAL, "null plan");
        cudaStream_t st = P->stream;
        const TreeDev& T = P->tree;
        int nb = T.nboxes;
        if (perm) {
            std::vector<int> h(P->n);
            CFMM_CUDA(cudaMemcpyAsync(h.data(), P->perm.get(), sizeof(int) * P->n, cudaMemcpyDeviceToHost, st));
            CFMM_CUDA(cudaStreamSynchronize(st));
            for (int64_t i = 0; i < P->n; ++i) perm[i] = h[i];
        }
        if (keys) CFMM_CUDA(cudaMemcpyAsync(keys, P->keys.get(), sizeof(uint64_t) * P->n, cudaMemcpyDeviceToHost, st));
        if (box_level) CFMM_CUDA(cudaMemcpyAsync(box_level, T.level.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        if (box_prefix) CFMM_CUDA(cudaMemcpyAsync(box_prefix, T.prefix.get(), sizeof(uint64_t) * nb, cudaMemcpyDeviceToHost, st));
        if (box_start) CFMM_CUDA(cudaMemcpyAsync(box_start, T.start.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        if (box_end) CFMM_CUDA(cudaMemcpyAsync(box_end, T.end.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        if (box_leaf) CFMM_CUDA(cudaMemcpyAsync(box_leaf, T.leaf.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        if (box_parent) CFMM_CUDA(cudaMemcpyAsync(box_parent, T.parent.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        if (center_re) CFMM_CUDA(cudaMemcpyAsync(center_re, T.cen_re.get(), sizeof(double) * nb * P->dim, cudaMemcpyDeviceToHost, st));
        if (center_im) CFMM_CUDA(cudaMemcpyAsync(center_im, T.cen_im.get(), sizeof(double) * nb * P->dim, cudaMemcpyDeviceToHost, st));
        CFMM_CUDA(cudaStreamSynchronize(st));
    });
}

int cfmm_plan_export_list(cfmm_plan_t P, int which, int64_t* offsets, int32_t* entries) {
    return guarded([&] {
        CFMM_REQUIRE(P, CFMM_EINVAL, "null plan");
        CFMM_REQUIRE(which >= 1 && which <= 4, CFMM_EINVAL, "which must be 1..4");
        const TreeDev& T = P->tree;
        int w = which - 1, nb = T.nboxes;
        cudaStream_t st = P->stream;
        if (offsets) {
            std::vector<int> h(nb + 1);
            CFMM_CUDA(cudaMemcpyAsync(h.data(), T.loff[w].get(), sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost, st));
            CFMM_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i <= nb; ++i) offsets[i] = h[i];
        }
        if (entries && T.llen[w] > 0)
            CFMM_CUDA(cudaMemcpyAsync(entries, T.lent[w].get(), sizeof(int) * T.llen[w], cudaMemcpyDeviceToHost, st));
        CFMM_CUDA(cudaStreamSynchronize(st));
    });
}

int cfmm_plan_set_timing(cfmm_plan_t P, int on) {
    return guarded([&] {
        CFMM_REQUIRE(P, CFMM_EINVAL, "null plan");
        CFMM_REQUIRE(on >= 0 && on <= 2, CFMM_EINVAL, "timing mode must be 0, 1 or 2");
        P->timing = on != 0;
        P->serial = on == 2;
    });
}

int cfmm_plan_timings(cfmm_plan_t P, double* t, int nsteps) {
    int rc = guarded([&] {
        CFMM_REQUIRE(P && t, CFMM_EINVAL, "null argument");
        for (int i = 0; i < nsteps && i < 9; ++i) t[i] = P->step_ms[i];
    });
    return rc == 0 ? 9 : rc;
}

}  // extern "C"
