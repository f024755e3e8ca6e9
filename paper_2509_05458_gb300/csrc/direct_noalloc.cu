// cfmm_direct_noalloc: the direct sum of cfmm_direct without any device
// memory allocation.
//
// Some callers cannot allocate device memory while they run: a host program
// that handed its whole device-memory budget to a pool up front (so a
// cudaMalloc from this library would fail), or a latency-critical loop in
// which cudaMalloc/cudaFree, which may synchronise the device, are not
// acceptable. For them this entry point keeps its scratch -- the SoA copies of
// the points and normals the kernel reads -- in a fixed array in device
// memory that is part of the loaded library (every GPU that loads the library
// holds it until the process exits), and calls no cudaMalloc, cudaFree or
// allocating library routine. The caller still passes the inputs and the
// output.
//
// Limits: m <= kNoAllocMaxSources sources and n <= kNoAllocMaxTargets targets.
// All calls share the one array: two calls whose work overlaps on the GPU
// (different streams, or different host threads without ordering) race on
// it. Every call overwrites the parts it reads, so nothing needs to start at
// zero. The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) and uploads the library's constant tables; make that
// first call before any stream capture.
#include <cmath>
#include <mutex>

#include "cfmm_special.cuh"
#include "kernels.cuh"

namespace cfmm {

constexpr int64_t kNoAllocMaxSources = 32768;
constexpr int64_t kNoAllocMaxTargets = 32768;
// src re, im, normal re, im: 4 * 3 * m ; trg re, im: 2 * 3 * n
constexpr int64_t kNoAllocScratchDoubles = 4 * 3 * kNoAllocMaxSources + 2 * 3 * kNoAllocMaxTargets;

static __device__ __align__(256) double g_direct_scratch[kNoAllocScratchDoubles];

// [cnt][dim] row-major -> [dim][cnt]
__global__ void k_aos_to_soa(const double* __restrict__ aos, int64_t cnt, int dim, double* __restrict__ soa) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    for (int a = 0; a < dim; ++a) soa[a * cnt + i] = aos[i * dim + a];
}

__global__ void k_scale_inplace(cd* __restrict__ v, int64_t cnt, cd s) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < cnt) v[i] = v[i] * s;
}

void launch_scale_inplace(cd* v, int64_t cnt, cd s, cudaStream_t st) {
    if (cnt <= 0) return;
    k_scale_inplace<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(v, cnt, s);
    CFMM_LAUNCHED();
}

// device address of the scratch array, looked up once per device
static double* scratch_address() {
    static std::mutex mu;
    static std::vector<double*> addr;
    int dev = 0;
    CFMM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_direct_scratch);
        if (e != cudaSuccess || !p)
            throw Error{CFMM_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
        addr[dev] = static_cast<double*>(p);
    }
    return addr[dev];
}

int direct_noalloc(int dim, int kernel, double k, const double* src_re, const double* src_im, const double* nrm_re,
                   const double* nrm_im, int64_t m, const double* trg_re, const double* trg_im, int64_t n,
                   const double* densities, int nrhs, double* out, void* stream) {
    CFMM_REQUIRE(dim == 2 || dim == 3, CFMM_EINVAL, "dim must be 2 or 3");
    int ker = kernel & 0xF;
    CFMM_REQUIRE(ker == CFMM_LAPLACE || ker == CFMM_HELMHOLTZ, CFMM_EINVAL, "bad kernel");
    CFMM_REQUIRE((kernel & ~(0xF | CFMM_SLP | CFMM_DLP | CFMM_GREEN_SCALE)) == 0, CFMM_EINVAL, "unknown kernel flags");
    CFMM_REQUIRE(ker == CFMM_LAPLACE || (std::isfinite(k) && k > 0.0), CFMM_EINVAL, "Helmholtz needs k > 0");
    CFMM_REQUIRE(m >= 1 && n >= 1 && nrhs >= 1, CFMM_EINVAL, "sizes must be positive");
    CFMM_REQUIRE(m <= kNoAllocMaxSources && n <= kNoAllocMaxTargets, CFMM_EINVAL,
                 "cfmm_direct_noalloc: at most 32768 sources and 32768 targets (fixed scratch array)");
    CFMM_REQUIRE(src_re && src_im && trg_re && trg_im && densities && out, CFMM_EINVAL, "null pointer");
    bool dlp = (kernel & CFMM_DLP) != 0;
    bool slp = (kernel & CFMM_SLP) != 0 || !dlp;
    CFMM_REQUIRE(!dlp || (nrm_re && nrm_im), CFMM_EINVAL, "double layer needs normals");
    // the first CUDA call of this entry point: everything above is host-only
    CFMM_REQUIRE(is_device_ptr(src_re) && is_device_ptr(trg_re) && is_device_ptr(densities) && is_device_ptr(out),
                 CFMM_EINVAL, "cfmm_direct_noalloc takes device pointers");
    ensure_device_tables();
    double* base = scratch_address();
    cudaStream_t st = (cudaStream_t)stream;
    double* sr = base;
    double* si = sr + 3 * kNoAllocMaxSources;
    double* nr = si + 3 * kNoAllocMaxSources;
    double* ni = nr + 3 * kNoAllocMaxSources;
    double* tr = ni + 3 * kNoAllocMaxSources;
    double* ti = tr + 3 * kNoAllocMaxTargets;
    auto soa = [&](const double* src, int64_t cnt, double* dst) {
        k_aos_to_soa<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(src, cnt, dim, dst);
        CFMM_LAUNCHED();
    };
    soa(src_re, m, sr);
    soa(src_im, m, si);
    soa(trg_re, n, tr);
    soa(trg_im, n, ti);
    if (dlp) {
        soa(nrm_re, m, nr);
        soa(nrm_im, m, ni);
    }
    int ncomp = (slp ? 1 : 0) + (dlp ? 1 : 0);
    const cd* d = reinterpret_cast<const cd*>(densities);
    KParams K{sr, si, dlp ? nr : nullptr, dlp ? ni : nullptr, tr, ti, m, n,
              slp ? d : nullptr, dlp ? d + (slp ? m : 0) : nullptr, ncomp * m, slp, dlp, k};
    launch_direct(dim, ker, K, reinterpret_cast<cd*>(out), nrhs, st);
    if (kernel & CFMM_GREEN_SCALE) launch_scale_inplace(reinterpret_cast<cd*>(out), n * nrhs, green_scale(dim, ker), st);
    return 0;
}

}  // namespace cfmm
