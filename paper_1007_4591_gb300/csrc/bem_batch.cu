// Many molecules at once, and the tuner of the octree leaf size and the
// expansion order.
//
// bem_batch_solve runs the full pipeline (right-hand side, GMRES, energy and
// the BIBEE bounds) for a set of independent meshes.  Each mesh owns a work
// stream and its K' product is a captured graph, so host worker threads that
// each drive one mesh keep several molecules' kernels in flight on the GPU
// at once; uneven sizes balance through a shared work counter (largest
// molecules first).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bem_internal.cuh"

using namespace bem;

extern "C" {

int bem_batch_solve(bem_mesh *const *meshes, int n, int threads, double *const *sigma, double *dG,
                    double *dG_cfa, double *dG_p, bem_solve_stats *stats) {
    if (!meshes || n < 0) {
        set_last_error("bem_batch_solve: bad arguments");
        return BEM_EINVAL;
    }
    if (n == 0) return BEM_OK;
    for (int i = 0; i < n; ++i)
        if (!meshes[i]) {
            set_last_error("bem_batch_solve: NULL mesh");
            return BEM_EINVAL;
        }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_last_error("bem_batch_solve: no CUDA device");
        return BEM_ECUDA;
    }
    // largest first
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        bem_mesh_info ia, ib;
        bem_mesh_info_get(meshes[a], &ia);
        bem_mesh_info_get(meshes[b], &ib);
        return ia.n_p > ib.n_p;
    });
    std::atomic<int> next(0);
    std::vector<int> rc(n, BEM_OK);
    std::vector<std::string> msg(n);
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= n) break;
            const int i = order[k];
            bem_mesh *m = meshes[i];
            bem_mesh_info info;
            bem_mesh_info_get(m, &info);
            double *sig = sigma ? sigma[i] : nullptr;
            double *own = nullptr;
            if (!sig) {
                if (cudaMalloc(&own, (size_t)info.n_p * sizeof(double)) != cudaSuccess) {
                    rc[i] = BEM_ENOMEM;
                    msg[i] = "batch: allocation failed";
                    continue;
                }
                sig = own;
            }
            bem_solve_stats st{};
            int r = bem_solve(m, nullptr, sig, &st);
            if (r != BEM_OK) msg[i] = bem_last_error();
            if (r == BEM_OK || r == BEM_ENOCONV) {
                double e = 0;
                int r2 = bem_energy(m, sig, &e, nullptr);
                if (dG) dG[i] = e;
                if (r2 == BEM_OK && dG_cfa) r2 = bem_bibee(m, BEM_BIBEE_CFA, nullptr, &dG_cfa[i]);
                if (r2 == BEM_OK && dG_p) r2 = bem_bibee(m, BEM_BIBEE_P, nullptr, &dG_p[i]);
                if (r2 != BEM_OK) {
                    r = r2;
                    msg[i] = bem_last_error();
                }
            }
            if (stats) stats[i] = st;
            rc[i] = r;
            if (own) cudaFree(own);
        }
    };
    const int nt = std::max(1, std::min(n, threads > 0 ? threads : 8));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto &t : pool) t.join();
    int worst = BEM_OK;
    for (int i = 0; i < n; ++i) {
        if (rc[i] != BEM_OK && rc[i] != BEM_ENOCONV) {
            set_last_error("molecule " + std::to_string(i) + ": " + msg[i]);
            return rc[i];
        }
        if (rc[i] == BEM_ENOCONV) worst = BEM_ENOCONV;
    }
    if (worst != BEM_OK) set_last_error("GMRES did not reach the tolerance for some molecules");
    return worst;
}

// Pick leaf_size in {32, 64, 128, 256} and p in {6, 8, 10} for one geometry:
// the fastest K' product whose relative error against a p = 12 product
// (on the right-hand side as input) is at most `target`.
int bem_autotune(const double *panels, int64_t n_p, const double *charges, int64_t n_c,
                 double eps_in, double eps_out, double target, bem_options *opt) {
    if (!opt || !panels || n_p <= 0 || !(target > 0)) {
        set_last_error("bem_autotune: bad arguments");
        return BEM_EINVAL;
    }
    bem_options base = *opt;
    base.depth = 0;
    bem_options ref = base;
    ref.p = 12;
    ref.leaf_size = 64;
    ref.graph = 0;
    bem_mesh *mr = nullptr;
    int r = bem_mesh_create(panels, n_p, charges, n_c, eps_in, eps_out, &ref, nullptr, &mr);
    if (r != BEM_OK) return r;
    double *x = nullptr, *yr = nullptr, *y = nullptr;
    if (cudaMalloc(&x, n_p * sizeof(double)) != cudaSuccess || cudaMalloc(&yr, n_p * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&y, n_p * sizeof(double)) != cudaSuccess) {
        bem_mesh_destroy(mr);
        cudaFree(x);
        cudaFree(yr);
        set_last_error("bem_autotune: allocation failed");
        return BEM_ENOMEM;
    }
    r = (n_c > 0) ? bem_rhs(mr, x) : BEM_OK;
    if (n_c == 0) {  // a smooth input without charges: the panels' z coordinate
        std::vector<double> h(n_p);
        std::vector<double> pan((size_t)n_p * 9);
        cudaPointerAttributes a;
        const bool dev_in = cudaPointerGetAttributes(&a, panels) == cudaSuccess &&
                            (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        cudaMemcpy(pan.data(), panels, pan.size() * sizeof(double),
                   dev_in ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
        for (int64_t i = 0; i < n_p; ++i) h[i] = (pan[9 * i + 2] + pan[9 * i + 5] + pan[9 * i + 8]) / 3.0;
        cudaMemcpy(x, h.data(), n_p * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (r == BEM_OK) r = bem_matvec(mr, x, yr);
    std::vector<double> hr(n_p), hy(n_p);
    if (r == BEM_OK) cudaMemcpy(hr.data(), yr, n_p * sizeof(double), cudaMemcpyDeviceToHost);
    bem_mesh_destroy(mr);
    double rn = 0;
    for (double v : hr) rn += v * v;
    rn = std::sqrt(rn);
    double best_t = 1e300, best_err = 1e300;
    int best_leaf = base.leaf_size, best_p = base.p;
    bool found = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int leaf : {32, 64, 128, 256}) {
        for (int p : {6, 8, 10}) {
            if (r != BEM_OK) break;
            bem_options c = base;
            c.leaf_size = leaf;
            c.p = p;
            bem_mesh *m = nullptr;
            r = bem_mesh_create(panels, n_p, charges, n_c, eps_in, eps_out, &c, nullptr, &m);
            if (r != BEM_OK) break;
            r = bem_matvec(m, x, y);
            float ms = 0;
            if (r == BEM_OK) {
                cudaEventRecord(e0, 0);
                for (int k = 0; k < 3; ++k) bem_matvec(m, x, y);
                cudaEventRecord(e1, 0);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                cudaMemcpy(hy.data(), y, n_p * sizeof(double), cudaMemcpyDeviceToHost);
            }
            bem_mesh_destroy(m);
            double d = 0;
            for (int64_t i = 0; i < n_p; ++i) d += (hy[i] - hr[i]) * (hy[i] - hr[i]);
            const double err = std::sqrt(d) / (rn > 0 ? rn : 1.0);
            if (err <= target && ms < best_t) {
                best_t = ms;
                best_leaf = leaf;
                best_p = p;
                found = true;
            }
            if (!found && err < best_err) {
                best_err = err;
                best_leaf = leaf;
                best_p = p;
            }
            if (err <= target) break;  // higher p at this leaf size is only slower
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(yr);
    cudaFree(y);
    if (r != BEM_OK) return r;
    opt->leaf_size = best_leaf;
    opt->p = best_p;
    opt->depth = 0;
    return BEM_OK;
}

}  // extern "C"
