// bem_normal_field_noalloc: the normal electric field of point charges at
// arbitrary points, for callers that cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc at the moment they need this product:
// code running inside another framework's memory pool that forbids outside
// allocations, a real-time loop that must not hit the allocator (an
// allocation can synchronise the device or fail under memory pressure), or
// a host that has handed all free device memory to someone else.  Those
// callers pass device buffers for every input and output; the only scratch
// the computation needs (the partial sums of the source splits) lives in one
// fixed array in this library's device image, so nothing is allocated here.
//
// Limits and sharing rules:
//  * the scratch holds BEM_NOALLOC_SCRATCH_FLOATS floats (8 MiB, held on
//    every device that loads the library until the process exits); a call
//    needs n_t x splits of them and is rejected with BEM_EINVAL when even one
//    split does not fit (n_t > BEM_NOALLOC_SCRATCH_FLOATS);
//  * every call on a device shares the one array and leaves its contents
//    behind; each call overwrites the part it reads, so no clearing is needed,
//    but calls that overlap on the GPU (different streams, or different host
//    threads) race on it and must be serialised by the caller;
//  * the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) and the device's SM count and keeps them; make
//    that first call outside any stream capture.
//  * every array must be device memory of the current device (or managed
//    memory); memory of another device is rejected.
#include <cmath>
#include <mutex>

#include "bem_internal.cuh"

namespace bem {

constexpr int64_t NOALLOC_FLOATS = (int64_t)1 << 21;  // = BEM_NOALLOC_SCRATCH_FLOATS
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

static std::mutex g_noalloc_mu;
static float *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
static int g_noalloc_sms[NOALLOC_MAX_DEVICES] = {};

// Set-up of the current device, once: the device address of the scratch
// array (host code cannot use the array's name as an address) and the SM
// count that sizes the source splits.
static float *noalloc_scratch(int dev, int *sms) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) throw Error(BEM_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        BEM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        int n = 0;
        BEM_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        g_noalloc_sms[dev] = n > 0 ? n : 1;
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *sms = g_noalloc_sms[dev];
    return g_noalloc_ptr[dev];
}

// field_i = sum_k q_k [-(t_i - x_k).n_i] / (4 pi |t_i - x_k|^3): FP32 pairs,
// per-split partial sums in the scratch array, FP64 reduction of the splits.
// Coordinates enter the FP32 arithmetic relative to the first target of the
// CTA (the shift is taken in FP64), so that the differences of nearby points
// keep their precision however far the system lies from the origin.
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_nf_partial(const double *tpos, const double *tnrm, int64_t nt, const double *ch, int64_t nc,
             int64_t chunk, float *part) {
    __shared__ float4 sh[NOALLOC_THREADS];
    const int64_t i0 = blockIdx.x * (int64_t)NOALLOC_THREADS;
    const int64_t i = i0 + threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.y * chunk, s1 = min(nc, s0 + chunk);
    const double ox = tpos[3 * i0], oy = tpos[3 * i0 + 1], oz = tpos[3 * i0 + 2];
    float x = 0, y = 0, z = 0, nx = 0, ny = 0, nz = 0;
    if (i < nt) {
        x = (float)(tpos[3 * i] - ox);
        y = (float)(tpos[3 * i + 1] - oy);
        z = (float)(tpos[3 * i + 2] - oz);
        nx = (float)tnrm[3 * i];
        ny = (float)tnrm[3 * i + 1];
        nz = (float)tnrm[3 * i + 2];
    }
    float outer = 0.f;
    for (int64_t b = s0; b < s1; b += NOALLOC_THREADS) {
        __syncthreads();
        const int64_t k = b + threadIdx.x;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < s1)
            r = make_float4((float)(ch[4 * k] - ox), (float)(ch[4 * k + 1] - oy), (float)(ch[4 * k + 2] - oz),
                            (float)ch[4 * k + 3]);
        sh[threadIdx.x] = r;
        __syncthreads();
        const int cnt = (int)min((int64_t)NOALLOC_THREADS, s1 - b);
        float acc = 0.f;
        for (int j = 0; j < cnt; ++j) {
            const float4 c = sh[j];
            const float dx = x - c.x, dy = y - c.y, dz = z - c.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 == 0.f) continue;
            const float ri = rsqrtf(r2);
            const float nd = fmaf(nx, dx, fmaf(ny, dy, nz * dz));
            acc = fmaf(c.w * nd, ri * ri * ri, acc);
        }
        outer += acc;
    }
    if (i < nt) part[(size_t)blockIdx.y * nt + i] = -outer;
}

__global__ void k_nf_reduce(const float *part, int nsplit, int64_t nt, double *field) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += (double)part[(size_t)k * nt + i];
    field[i] = s / FOUR_PI;
}

// Device memory of device `dev`, or managed memory.
static bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace bem

using namespace bem;

extern "C" int bem_normal_field_noalloc(const double *targets, const double *normals, int64_t n_t,
                                        const double *charges, int64_t n_c, double *field,
                                        void *stream) {
    try {
        if (n_t < 0 || n_c < 0) throw Error(BEM_EINVAL, "bem_normal_field_noalloc: negative size");
        if (n_t == 0) return BEM_OK;
        if (n_t > NOALLOC_FLOATS)
            throw Error(BEM_EINVAL, "bem_normal_field_noalloc: n_t = " + std::to_string(n_t) +
                                        " exceeds the scratch limit of " + std::to_string(NOALLOC_FLOATS) +
                                        " targets (use bem_mesh_create + bem_rhs instead)");
        if (!targets || !normals || !field || (n_c > 0 && !charges))
            throw Error(BEM_EINVAL, "bem_normal_field_noalloc: NULL array");
        int dev = 0;
        BEM_CUDA(cudaGetDevice(&dev));
        const struct { const void *p; const char *name; } args[] = {
            {targets, "targets"}, {normals, "normals"}, {field, "field"}, {n_c > 0 ? charges : targets, "charges"}};
        for (const auto &a : args)
            if (!on_device(a.p, dev))
                throw Error(BEM_EINVAL, std::string("bem_normal_field_noalloc: ") + a.name +
                                            " must be device memory of the current device");
        cudaStream_t s = (cudaStream_t)stream;
        int sms = 1;
        float *part = noalloc_scratch(dev, &sms);
        const int tblocks = cdiv(n_t, NOALLOC_THREADS);
        int64_t nsplit = 1;
        if (n_c > 0) {
            // about 8 CTAs per SM, splits of at least 4096 charges
            nsplit = std::max<int64_t>(1, std::min<int64_t>(cdiv(n_c, 4096), std::max(1, 8 * sms / tblocks)));
            nsplit = std::min<int64_t>(nsplit, NOALLOC_FLOATS / n_t);
            nsplit = std::min<int64_t>(nsplit, 65535);
        }
        int64_t chunk = n_c > 0 ? (n_c + nsplit - 1) / nsplit : 1;
        chunk = ((chunk + NOALLOC_THREADS - 1) / NOALLOC_THREADS) * NOALLOC_THREADS;
        if (n_c > 0) nsplit = (n_c + chunk - 1) / chunk;
        if (n_c == 0) {
            BEM_CUDA(cudaMemsetAsync(field, 0, n_t * sizeof(double), s));
            return BEM_OK;
        }
        dim3 grid(tblocks, (unsigned)nsplit);
        k_nf_partial<<<grid, NOALLOC_THREADS, 0, s>>>(targets, normals, n_t, charges, n_c, chunk, part);
        BEM_CHECK_LAUNCH();
        k_nf_reduce<<<cdiv(n_t, 256), 256, 0, s>>>(part, (int)nsplit, n_t, field);
        BEM_CHECK_LAUNCH();
        return BEM_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return BEM_ECUDA;
    }
}
