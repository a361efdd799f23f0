// Panel geometry, Morton ordering, octree and interaction lists (Sec. 2.3).
//
// Everything runs on the device: per-panel geometry and quadrature points,
// 63-bit Morton keys, radix sort of every point set, the uniform-depth octree
// ("divided ... until the finest level of refinement", Sec. 2.3) as sorted
// non-empty cells per level, the P2P neighbour list (the 26 adjacent cells
// plus the cell itself) and the M2L interaction list ("cells whose parents
// are neighbors of the given cell's parent, and yet not directly adjacent to
// the given cell", Sec. 2.3).

#include <algorithm>
#include <cmath>
#include <vector>

#include "bem_internal.cuh"

namespace bem {

// ------------------------------------------------------------------ quadrature
// Degree-5 seven-point triangle rule (Radon 1948; Stroud 1971, T2:5-1):
// centroid with weight 9/40; permutations of (a, a, 1-2a), a = (6-sqrt15)/21,
// weight (155-sqrt15)/1200; permutations of (b, b, 1-2b), b = (6+sqrt15)/21,
// weight (155+sqrt15)/1200.  With nq = 1 the centroid alone (weight 1).
__constant__ double c_qbary[7][3];
__constant__ double c_qw[7];

static void upload_rule(int nq) {
    double bary[7][3] = {}, w[7] = {};
    if (nq == 1) {
        bary[0][0] = bary[0][1] = bary[0][2] = 1.0 / 3.0;
        w[0] = 1.0;
    } else {
        const double r15 = std::sqrt(15.0);
        const double a = (6.0 - r15) / 21.0, b = (6.0 + r15) / 21.0;
        const double wa = (155.0 - r15) / 1200.0, wb = (155.0 + r15) / 1200.0;
        double pts[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                            {a, a, 1 - 2 * a}, {a, 1 - 2 * a, a}, {1 - 2 * a, a, a},
                            {b, b, 1 - 2 * b}, {b, 1 - 2 * b, b}, {1 - 2 * b, b, b}};
        double ww[7] = {9.0 / 40, wa, wa, wa, wb, wb, wb};
        for (int q = 0; q < 7; ++q) {
            for (int k = 0; k < 3; ++k) bary[q][k] = pts[q][k];
            w[q] = ww[q];
        }
    }
    BEM_CUDA(cudaMemcpyToSymbol(c_qbary, bary, sizeof(bary)));
    BEM_CUDA(cudaMemcpyToSymbol(c_qw, w, sizeof(w)));
}

// -------------------------------------------------------------- Morton keys
__host__ __device__ inline uint64_t spread_bits(uint32_t v) {
    uint64_t x = v & 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ inline uint32_t compact_bits(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}
__host__ __device__ inline uint64_t morton3(uint32_t i, uint32_t j, uint32_t k) {
    return spread_bits(i) | (spread_bits(j) << 1) | (spread_bits(k) << 2);
}
__host__ __device__ inline void demorton3(uint64_t key, int &i, int &j, int &k) {
    i = (int)compact_bits(key);
    j = (int)compact_bits(key >> 1);
    k = (int)compact_bits(key >> 2);
}

struct Root {
    double lo[3];
    double inv_side;
};

__device__ inline uint64_t point_key(const Root &r, double x, double y, double z) {
    const double scale = (double)(1u << MORTON_BITS) * r.inv_side;
    const int mx = (1 << MORTON_BITS) - 1;
    int i = (int)floor((x - r.lo[0]) * scale);
    int j = (int)floor((y - r.lo[1]) * scale);
    int k = (int)floor((z - r.lo[2]) * scale);
    i = min(max(i, 0), mx);
    j = min(max(j, 0), mx);
    k = min(max(k, 0), mx);
    return morton3((uint32_t)i, (uint32_t)j, (uint32_t)k);
}

// ---------------------------------------------------------------- kernels
__global__ void k_bbox(const double *d, int64_t n, int stride, double *part) {
    __shared__ double sh[6][256];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            double v = d[i * stride + k];
            lo[k] = fmin(lo[k], v);
            hi[k] = fmax(hi[k], v);
        }
    }
    for (int k = 0; k < 3; ++k) {
        sh[k][threadIdx.x] = lo[k];
        sh[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k) {
                sh[k][threadIdx.x] = fmin(sh[k][threadIdx.x], sh[k][threadIdx.x + s]);
                sh[3 + k][threadIdx.x] = fmax(sh[3 + k][threadIdx.x], sh[3 + k][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[blockIdx.x * 6 + k] = sh[k][0];
}

void compute_bbox(const double *d, int64_t n, int stride, double *lo, double *hi, cudaStream_t s) {
    const int nb = 256;
    DArray<double> part;
    part.alloc(nb * 6);
    k_bbox<<<nb, 256, 0, s>>>(d, n, stride, part);
    BEM_CHECK_LAUNCH();
    std::vector<double> h(nb * 6);
    BEM_CUDA(cudaMemcpyAsync(h.data(), part.p, nb * 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; ++k) { lo[k] = 1e300; hi[k] = -1e300; }
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], h[b * 6 + k]);
            hi[k] = std::max(hi[k], h[b * 6 + 3 + k]);
        }
}

// Geometry of every panel (original order): centroid, unit normal, area and
// quadrature points y_jq = sum_k bary_qk v_k with weights A_j w_q (Sec. 2.1).
__global__ void k_panel_geometry(const double *pan, int64_t np, int nq, double *cen, double *nrm,
                                 double *area, double *qp, double *qw, int *bad) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const double *v = pan + 9 * j;
    double e1[3], e2[3];
    bool fin = true;
    for (int k = 0; k < 9; ++k) fin = fin && isfinite(v[k]);
    for (int k = 0; k < 3; ++k) {
        e1[k] = v[3 + k] - v[k];
        e2[k] = v[6 + k] - v[k];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1];
    double cy = e1[2] * e2[0] - e1[0] * e2[2];
    double cz = e1[0] * e2[1] - e1[1] * e2[0];
    double len = sqrt(cx * cx + cy * cy + cz * cz);
    // relative test: with fused multiply-adds an exactly degenerate triangle
    // leaves a cross product at the rounding level, not exactly zero
    const double e1n = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    const double e2n = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    if (!fin || !(len > 1e-12 * e1n * e2n) || !isfinite(len)) {
        atomicExch(bad, 1);
        len = 1.0;
    }
    double A = 0.5 * len;
    area[j] = A;
    nrm[3 * j] = cx / len;
    nrm[3 * j + 1] = cy / len;
    nrm[3 * j + 2] = cz / len;
    double c[3];
    for (int k = 0; k < 3; ++k) {
        c[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
        cen[3 * j + k] = c[k];
    }
    for (int q = 0; q < nq; ++q) {
        for (int k = 0; k < 3; ++k) {
            double y = c_qbary[q][0] * v[k] + c_qbary[q][1] * v[3 + k] + c_qbary[q][2] * v[6 + k];
            // the rule's centroid node is the collocation point itself
            if (q == 0) y = c[k];
            qp[(j * nq + q) * 3 + k] = y;
        }
        qw[j * nq + q] = A * c_qw[q];
    }
}

__global__ void k_keys(const double *pts, int64_t n, int stride, Root r, uint64_t *key, int *idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *x = pts + i * stride;
    key[i] = point_key(r, x[0], x[1], x[2]);
    idx[i] = (int)i;
}

__global__ void k_check_charges(const double *ch, int64_t n, int *bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 4; ++k)
        if (!isfinite(ch[4 * i + k])) atomicExch(bad, 1);
}

// Winding number of the surface around each charge, times 4 pi: the sum of
// the solid angles its panels subtend (triple-product formula for a
// triangle's solid angle), -4 pi for a point enclosed by a closed surface
// with outward normals and 0 outside it.  Each thread sums one charge over
// a chunk of panels (FP32: the two values are far apart).
__global__ void k_winding(const double *pan, int64_t np, const double *ch, int64_t nc, int64_t chunk,
                          double *wind) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const float px = (float)ch[4 * k], py = (float)ch[4 * k + 1], pz = (float)ch[4 * k + 2];
    const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(np, j0 + chunk);
    float acc = 0.f;
    for (int64_t j = j0; j < j1; ++j) {
        const double *v = pan + 9 * j;
        float r[3][3], l[3];
        for (int a = 0; a < 3; ++a) {
            r[a][0] = (float)v[3 * a] - px;
            r[a][1] = (float)v[3 * a + 1] - py;
            r[a][2] = (float)v[3 * a + 2] - pz;
            l[a] = sqrtf(r[a][0] * r[a][0] + r[a][1] * r[a][1] + r[a][2] * r[a][2]);
        }
        const float cx = r[1][1] * r[2][2] - r[1][2] * r[2][1], cy = r[1][2] * r[2][0] - r[1][0] * r[2][2],
                    cz = r[1][0] * r[2][1] - r[1][1] * r[2][0];
        const float trip = r[0][0] * cx + r[0][1] * cy + r[0][2] * cz;
        auto d = [&](int a, int b) { return r[a][0] * r[b][0] + r[a][1] * r[b][1] + r[a][2] * r[b][2]; };
        const float den = l[0] * l[1] * l[2] + d(0, 1) * l[2] + d(0, 2) * l[1] + d(1, 2) * l[0];
        acc += -2.f * atan2f(trip, den);  // positive seen from the side the normal points to
    }
    atomicAdd(wind + k, (double)acc);
}

// Level histogram: pair (i-1, i) of sorted keys separates cells at every
// level >= 21 - floor(hibit(key_i ^ key_{i-1}) / 3).
__global__ void k_level_hist(const uint64_t *key, int64_t n, unsigned long long *hist) {
    __shared__ unsigned long long sh[MORTON_BITS + 2];
    if (threadIdx.x < MORTON_BITS + 2) sh[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = key[i] ^ key[i - 1];
        if (x) {
            int hb = 63 - __clzll((long long)x);
            int l0 = MORTON_BITS - hb / 3;
            atomicAdd(&sh[l0], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < MORTON_BITS + 2) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

template <class T>
__global__ void k_gather_rows(const T *src, const int *perm, T *dst, int64_t n, int w) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = perm[i];
    for (int k = 0; k < w; ++k) dst[i * w + k] = src[s * w + k];
}

__global__ void k_split_charges(const double *ch, const int *perm, int64_t n, double *xyz,
                                double *q) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = perm[i];
    xyz[3 * i] = ch[4 * s];
    xyz[3 * i + 1] = ch[4 * s + 1];
    xyz[3 * i + 2] = ch[4 * s + 2];
    q[i] = ch[4 * s + 3];
}

__global__ void k_inverse_perm(const int *perm, int *rank, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) rank[perm[i]] = (int)i;
}

__global__ void k_qp_of_panel(const int *cen_perm, const int *invq, int nq, int64_t np, int *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np * nq) return;
    const int64_t j = i / nq, q = i - j * nq;
    out[i] = invq[(int64_t)cen_perm[j] * nq + q];
}

__global__ void k_qp_panel(const int *qperm, const int *rank, int nq, int *qpanel, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) qpanel[i] = rank[qperm[i] / nq];
}

// Leaf-relative records: coordinates minus the centre of the point's own leaf.
struct LeafGeom {
    double lo[3];
    double h;   // leaf cell size
    int shift;  // 3 * (21 - L)
};

__device__ inline void leaf_center(const LeafGeom &g, uint64_t key, double *c) {
    int i, j, k;
    demorton3(key >> g.shift, i, j, k);
    c[0] = g.lo[0] + (i + 0.5) * g.h;
    c[1] = g.lo[1] + (j + 0.5) * g.h;
    c[2] = g.lo[2] + (k + 0.5) * g.h;
}

__global__ void k_rel_records(const double *pos, const double *w, const double *nrm,
                              const uint64_t *key, int64_t n, LeafGeom g, float4 *r32,
                              double4 *r64, float4 *n32, double4 *n64) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double c[3];
    leaf_center(g, key[i], c);
    double x = pos[3 * i] - c[0], y = pos[3 * i + 1] - c[1], z = pos[3 * i + 2] - c[2];
    double ww = w ? w[i] : 0.0;
    if (r32) r32[i] = make_float4((float)x, (float)y, (float)z, (float)ww);
    if (r64) r64[i] = make_double4(x, y, z, ww);
    if (nrm) {
        double a = nrm[3 * i], b = nrm[3 * i + 1], cc = nrm[3 * i + 2];
        if (n32) n32[i] = make_float4((float)a, (float)b, (float)cc, 0.f);
        if (n64) n64[i] = make_double4(a, b, cc, 0.0);
    }
}

// ------------------------------------------------------------ tree kernels
__global__ void k_prefix(const uint64_t *key, int64_t n, int shift, uint64_t *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = key[i] >> shift;
}

__global__ void k_parent_flags(const uint64_t *ck, int n, uint64_t *pk, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t a = ck[i] >> 3;
    pk[i] = a;
    flag[i] = (i == 0 || (ck[i - 1] >> 3) != a) ? 1 : 0;
}

__global__ void k_parent_fill(const uint64_t *pk, const int *flag, const int *pidx, int n,
                              uint64_t *pkeys, int *child_first) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    int p = pidx[i] - 1;
    pkeys[p] = pk[i];
    child_first[p] = i;
}

__global__ void k_cells_level(const uint64_t *lkeys, int cnt, int level, int off, int child_off,
                              int child_cnt, const int *child_first, const int *pidx_child,
                              int parent_off, uint64_t *key, int4 *ijk, int *cbeg, int *cend,
                              int *parent) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    uint64_t k = lkeys[i];
    int a, b, c;
    demorton3(k, a, b, c);
    key[off + i] = k;
    ijk[off + i] = make_int4(a, b, c, level);
    if (child_first) {
        int f = child_first[i];
        int e = (i + 1 < cnt) ? child_first[i + 1] : child_cnt;
        cbeg[off + i] = child_off + f;
        cend[off + i] = child_off + e;
    } else {
        cbeg[off + i] = -1;
        cend[off + i] = -1;
    }
    parent[off + i] = (pidx_child != nullptr) ? parent_off + pidx_child[i] - 1 : -1;
}

__device__ inline int find_key(const uint64_t *keys, int lo, int hi, uint64_t k) {
    // index of k in sorted keys[lo, hi), or -1
    const int end = hi;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && keys[lo] == k) ? lo : -1;
}

__global__ void k_leaf_csr(const uint64_t *setkey, int64_t n, int shift, const uint64_t *leafkey,
                           int nleaf, int *beg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nleaf) return;
    if (i == nleaf) {
        beg[i] = (int)n;
        return;
    }
    uint64_t k = leafkey[i];
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((setkey[mid] >> shift) < k) lo = mid + 1;
        else hi = mid;
    }
    beg[i] = (int)lo;
}

// P2P neighbour list: the leaves within ws cells (the adjacent ones for
// ws = 1, and the leaf itself) that exist.
template <bool FILL>
__global__ void k_nbr(const uint64_t *key, const int4 *ijk, int leaf0, int nleaf, int L, int ws,
                      const int *off, int *cnt_or_list) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    int4 c = ijk[leaf0 + t];
    int lim = 1 << L;
    int n = 0;
    int base = FILL ? off[t] : 0;
    for (int dx = -ws; dx <= ws; ++dx)
        for (int dy = -ws; dy <= ws; ++dy)
            for (int dz = -ws; dz <= ws; ++dz) {
                int a = c.x + dx, b = c.y + dy, e = c.z + dz;
                if (a < 0 || b < 0 || e < 0 || a >= lim || b >= lim || e >= lim) continue;
                int f = find_key(key, leaf0, leaf0 + nleaf, morton3(a, b, e));
                if (f < 0) continue;
                if (FILL) cnt_or_list[base + n] = f - leaf0;
                ++n;
            }
    if (!FILL) cnt_or_list[t] = n;
}

// M2L list of cell t (level >= 2): children of the neighbours of t's parent
// (the cells within ws of it) that are not neighbours of t.  With
// R = 2 ws + 1 and W = 2 R + 1 the offset class is
// (dx+R)*W*W + (dy+R)*W + (dz+R), (dx,dy,dz) = ijk_source - ijk_target in [-R,R]^3.
template <bool FILL>
__global__ void k_m2l(const uint64_t *key, const int4 *ijk, const int *parent, const int *cbeg,
                      const int *cend, const int *lvl_off, int first, int last, int ws, const int *off,
                      int *cnt, int *src, int *ofs) {
    int t = first + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= last) return;
    int4 c = ijk[t];
    int l = c.w;
    int n = 0;
    const int R = 2 * ws + 1, W = 2 * R + 1;
    if (l >= 2) {
        int P = parent[t];
        int4 pc = ijk[P];
        int lim = 1 << (l - 1);
        int plo = lvl_off[l - 1], phi = lvl_off[l];
        int base = FILL ? off[t] : 0;
        for (int dx = -ws; dx <= ws; ++dx)
            for (int dy = -ws; dy <= ws; ++dy)
                for (int dz = -ws; dz <= ws; ++dz) {
                    int a = pc.x + dx, b = pc.y + dy, e = pc.z + dz;
                    if (a < 0 || b < 0 || e < 0 || a >= lim || b >= lim || e >= lim) continue;
                    int f = find_key(key, plo, phi, morton3(a, b, e));
                    if (f < 0) continue;
                    for (int s = cbeg[f]; s < cend[f]; ++s) {
                        int4 sc = ijk[s];
                        int ddx = sc.x - c.x, ddy = sc.y - c.y, ddz = sc.z - c.z;
                        if (abs(ddx) <= ws && abs(ddy) <= ws && abs(ddz) <= ws) continue;
                        if (FILL) {
                            src[base + n] = s;
                            ofs[base + n] = ((ddx + R) * W + (ddy + R)) * W + (ddz + R);
                        }
                        ++n;
                    }
                }
    }
    if (!FILL) cnt[t] = n;
}

__global__ void k_count_pairs(const int *tbeg, const int *sbeg, const int *nbr_off, const int *nbr,
                              int nleaf, unsigned long long *out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (t < nleaf) {
        long long nt = tbeg[t + 1] - tbeg[t];
        long long ns = 0;
        for (int e = nbr_off[t]; e < nbr_off[t + 1]; ++e) {
            int s = nbr[e];
            ns += sbeg[s + 1] - sbeg[s];
        }
        v = (unsigned long long)(nt * ns);
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, v);
}

// ----------------------------------------------------------- host helpers
// Morton sort of (key, index) pairs over the keys' 63 bits (stable).
static void sort_pairs(uint64_t *k_in, int *v_in, uint64_t *k_out, int *v_out, int64_t n, cudaStream_t s) {
    radix_sort_u64(k_in, v_in, k_out, v_out, n, 3 * MORTON_BITS, s);
}

void sort_pairs_int(const int *k_in, const int *v_in, int *k_out, int *v_out, int64_t n, int bits,
                    cudaStream_t s) {
    radix_sort_u32(reinterpret_cast<const uint32_t *>(k_in), v_in, reinterpret_cast<uint32_t *>(k_out), v_out, n,
                   bits, s);
}

static void scan_exclusive(const int *in, int *out, int n, cudaStream_t s) { scan_exclusive_i32(in, out, n, s); }

static void scan_inclusive(const int *in, int *out, int n, cudaStream_t s) { scan_inclusive_i32(in, out, n, s); }

template <class T>
static T to_host(const T *d, cudaStream_t s) {
    T v;
    BEM_CUDA(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    return v;
}

struct SetKeys {
    const uint64_t *key = nullptr;
    int64_t n = 0;
};

// Build the octree over up to three sorted point sets at leaf level L.
static void build_tree(Mesh &m, Tree &t, SetKeys cen, SetKeys qp, SetKeys chg, int ws) {
    cudaStream_t s = m.stream;
    const int L = m.L;
    t.ws = ws;
    const int shift = 3 * (MORTON_BITS - L);
    const int64_t total = cen.n + qp.n + chg.n;
    t.L = L;
    t.has_cen = cen.n > 0;
    t.has_qp = qp.n > 0;
    t.has_chg = chg.n > 0;
    const int TB = 256;

    // 1. leaf keys = sorted unique leaf prefixes of all sets
    DArray<uint64_t> pref, pref_sorted;
    pref.alloc(total);
    pref_sorted.alloc(total);
    int64_t o = 0;
    for (SetKeys sk : {cen, qp, chg}) {
        if (sk.n == 0) continue;
        k_prefix<<<cdiv(sk.n, TB), TB, 0, s>>>(sk.key, sk.n, shift, pref.p + o);
        BEM_CHECK_LAUNCH();
        o += sk.n;
    }
    radix_sort_u64(pref.p, nullptr, pref_sorted.p, nullptr, total, 3 * MORTON_BITS, s);
    const int nleaf = (int)unique_sorted_u64(pref_sorted.p, pref.p, total, s);

    // 2. levels bottom-up
    std::vector<DArray<uint64_t>> lkeys(L + 1);
    std::vector<DArray<int>> child_first(L + 1), pidx(L + 1);
    std::vector<int> cnt(L + 1);
    lkeys[L].alloc(nleaf);
    BEM_CUDA(cudaMemcpyAsync(lkeys[L].p, pref.p, nleaf * sizeof(uint64_t),
                             cudaMemcpyDeviceToDevice, s));
    cnt[L] = nleaf;
    for (int l = L - 1; l >= 0; --l) {
        int nch = cnt[l + 1];
        DArray<uint64_t> pk;
        DArray<int> flag;
        pk.alloc(nch);
        flag.alloc(nch);
        pidx[l + 1].alloc(nch);
        k_parent_flags<<<cdiv(nch, TB), TB, 0, s>>>(lkeys[l + 1].p, nch, pk.p, flag.p);
        BEM_CHECK_LAUNCH();
        scan_inclusive(flag.p, pidx[l + 1].p, nch, s);
        int np_ = to_host(pidx[l + 1].p + nch - 1, s);
        cnt[l] = np_;
        lkeys[l].alloc(np_);
        child_first[l].alloc(np_);
        k_parent_fill<<<cdiv(nch, TB), TB, 0, s>>>(pk.p, flag.p, pidx[l + 1].p, nch, lkeys[l].p,
                                                   child_first[l].p);
        BEM_CHECK_LAUNCH();
        BEM_CUDA(cudaStreamSynchronize(s));
    }
    t.lvl_off.assign(L + 2, 0);
    for (int l = 0; l <= L; ++l) t.lvl_off[l + 1] = t.lvl_off[l] + cnt[l];
    t.ncell = t.lvl_off[L + 1];
    t.nleaf = nleaf;
    t.leaf0 = t.lvl_off[L];
    t.key.alloc(t.ncell);
    t.ijk.alloc(t.ncell);
    t.parent.alloc(t.ncell);
    t.child_beg.alloc(t.ncell);
    t.child_end.alloc(t.ncell);
    for (int l = 0; l <= L; ++l) {
        const int *cf = (l < L) ? child_first[l].p : nullptr;
        const int *pi = (l > 0) ? pidx[l].p : nullptr;
        int coff = (l < L) ? t.lvl_off[l + 1] : 0;
        int ccnt = (l < L) ? cnt[l + 1] : 0;
        int poff = (l > 0) ? t.lvl_off[l - 1] : 0;
        k_cells_level<<<cdiv(cnt[l], TB), TB, 0, s>>>(lkeys[l].p, cnt[l], l, t.lvl_off[l], coff,
                                                      ccnt, cf, pi, poff, t.key.p, t.ijk.p,
                                                      t.child_beg.p, t.child_end.p, t.parent.p);
        BEM_CHECK_LAUNCH();
    }

    // 3. leaf CSR of every set
    auto csr = [&](SetKeys sk, DArray<int> &beg) {
        beg.alloc(nleaf + 1);
        if (sk.n == 0) {
            BEM_CUDA(cudaMemsetAsync(beg.p, 0, (nleaf + 1) * sizeof(int), s));
            return;
        }
        k_leaf_csr<<<cdiv(nleaf + 1, TB), TB, 0, s>>>(sk.key, sk.n, shift, t.key.p + t.leaf0, nleaf,
                                                     beg.p);
        BEM_CHECK_LAUNCH();
    };
    csr(cen, t.cen_beg);
    csr(qp, t.qp_beg);
    csr(chg, t.chg_beg);

    // 4. P2P neighbour lists
    {
        DArray<int> c;
        c.alloc(nleaf + 1);
        BEM_CUDA(cudaMemsetAsync(c.p, 0, (nleaf + 1) * sizeof(int), s));
        k_nbr<false><<<cdiv(nleaf, TB), TB, 0, s>>>(t.key.p, t.ijk.p, t.leaf0, nleaf, L, ws, nullptr, c.p);
        BEM_CHECK_LAUNCH();
        t.nbr_off.alloc(nleaf + 1);
        scan_exclusive(c.p, t.nbr_off.p, nleaf + 1, s);
        t.nnbr = to_host(t.nbr_off.p + nleaf, s);
        t.nbr.alloc(t.nnbr);
        k_nbr<true><<<cdiv(nleaf, TB), TB, 0, s>>>(t.key.p, t.ijk.p, t.leaf0, nleaf, L, ws, t.nbr_off.p,
                                                   t.nbr.p);
        BEM_CHECK_LAUNCH();
    }
    // 5. M2L lists (levels >= 2)
    {
        DArray<int> loff;
        loff.alloc(L + 2);
        BEM_CUDA(cudaMemcpyAsync(loff.p, t.lvl_off.data(), (L + 2) * sizeof(int),
                                 cudaMemcpyHostToDevice, s));
        DArray<int> c;
        c.alloc(t.ncell + 1);
        BEM_CUDA(cudaMemsetAsync(c.p, 0, (t.ncell + 1) * sizeof(int), s));
        k_m2l<false><<<cdiv(t.ncell, TB), TB, 0, s>>>(t.key.p, t.ijk.p, t.parent.p, t.child_beg.p,
                                                      t.child_end.p, loff.p, 0, t.ncell, ws, nullptr,
                                                      c.p, nullptr, nullptr);
        BEM_CHECK_LAUNCH();
        t.m2l_off.alloc(t.ncell + 1);
        scan_exclusive(c.p, t.m2l_off.p, t.ncell + 1, s);
        t.nm2l = to_host(t.m2l_off.p + t.ncell, s);
        t.m2l_src.alloc(t.nm2l);
        t.m2l_ofs.alloc(t.nm2l);
        k_m2l<true><<<cdiv(t.ncell, TB), TB, 0, s>>>(t.key.p, t.ijk.p, t.parent.p, t.child_beg.p,
                                                     t.child_end.p, loff.p, 0, t.ncell, ws, t.m2l_off.p,
                                                     nullptr, t.m2l_src.p, t.m2l_ofs.p);
        BEM_CHECK_LAUNCH();
        BEM_CUDA(cudaStreamSynchronize(s));
    }
    // 6. exact near-field pair count (centroid targets x quadrature sources)
    if (t.has_cen && t.has_qp) {
        DArray<unsigned long long> acc;
        acc.alloc(1);
        BEM_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), s));
        k_count_pairs<<<cdiv(nleaf, TB), TB, 0, s>>>(t.cen_beg.p, t.qp_beg.p, t.nbr_off.p, t.nbr.p,
                                                     nleaf, acc.p);
        BEM_CHECK_LAUNCH();
        t.p2p_pairs_cq = (int64_t)to_host(acc.p, s);
    }
}

size_t Tree::bytes() const {
    return g_out.bytes() + g_in.bytes() + g_chunk.bytes() + p2p_order.bytes() + tc_super.bytes() +
           p2p_hdr[0].bytes() + p2p_hdr[1].bytes() + p2p_rec[0].bytes() + p2p_rec[1].bytes() +
           key.bytes() + ijk.bytes() + parent.bytes() + child_beg.bytes() + child_end.bytes() +
           cen_beg.bytes() + qp_beg.bytes() + chg_beg.bytes() + nbr_off.bytes() + nbr.bytes() +
           m2l_off.bytes() + m2l_src.bytes() + m2l_ofs.bytes() + p2m_seg_beg.bytes() + p2m_seg_panel.bytes() +
           p2m_seg_f.bytes() + p2m_seg_d.bytes();
}

TreeView view(const Tree &t) {
    TreeView v;
    v.L = t.L;
    v.ncell = t.ncell;
    v.nleaf = t.nleaf;
    v.leaf0 = t.leaf0;
    v.ijk = t.ijk.p;
    v.parent = t.parent.p;
    v.child_beg = t.child_beg.p;
    v.child_end = t.child_end.p;
    v.cen_beg = t.cen_beg.p;
    v.qp_beg = t.qp_beg.p;
    v.chg_beg = t.chg_beg.p;
    v.nbr_off = t.nbr_off.p;
    v.nbr = t.nbr.p;
    v.m2l_off = t.m2l_off.p;
    v.m2l_src = t.m2l_src.p;
    v.m2l_ofs = t.m2l_ofs.p;
    v.p2p_order = t.p2p_order.p;
    v.seg_beg = t.p2m_seg_p >= 0 ? t.p2m_seg_beg.p : nullptr;
    v.seg_panel = t.p2m_seg_panel.p;
    v.seg_f = t.p2m_seg_f.p;
    v.seg_d = t.p2m_seg_d.p;
    v.seg_p = t.p2m_seg_p;
    return v;
}

static LeafGeom leaf_geom(const Mesh &m) {
    LeafGeom g;
    for (int k = 0; k < 3; ++k) g.lo[k] = m.root_min[k];
    g.h = m.side / (double)(1 << m.L);
    g.shift = 3 * (MORTON_BITS - m.L);
    return g;
}

static Root root_of(const Mesh &m) {
    Root r;
    for (int k = 0; k < 3; ++k) r.lo[k] = m.root_min[k];
    r.inv_side = 1.0 / m.side;
    return r;
}

// Sort the charges and (re)build the charge tree.
static void build_charges(Mesh &m, const double *d_charges) {
    cudaStream_t s = m.stream;
    const int TB = 256;
    const int64_t nc = m.nc;
    m.chg_perm.release();
    m.chgg64.release();
    m.q64.release();
    m.chg32.release();
    m.chg64r.release();
    m.chg_key.release();
    if (nc > 0) {
        DArray<uint64_t> k0;
        DArray<int> i0;
        k0.alloc(nc);
        i0.alloc(nc);
        m.chg_key.alloc(nc);
        m.chg_perm.alloc(nc);
        k_keys<<<cdiv(nc, TB), TB, 0, s>>>(d_charges, nc, 4, root_of(m), k0.p, i0.p);
        BEM_CHECK_LAUNCH();
        sort_pairs(k0.p, i0.p, m.chg_key.p, m.chg_perm.p, nc, s);
        m.chgg64.alloc(nc * 3);
        m.q64.alloc(nc);
        k_split_charges<<<cdiv(nc, TB), TB, 0, s>>>(d_charges, m.chg_perm.p, nc, m.chgg64.p, m.q64.p);
        BEM_CHECK_LAUNCH();
        LeafGeom g = leaf_geom(m);
        if (m.opt.precision == BEM_MIXED) m.chg32.alloc(nc);
        else m.chg64r.alloc(nc);
        k_rel_records<<<cdiv(nc, TB), TB, 0, s>>>(m.chgg64.p, m.q64.p, nullptr, m.chg_key.p, nc, g,
                                                  m.chg32.p, m.chg64r.p, nullptr, nullptr);
        BEM_CHECK_LAUNCH();
        BEM_CUDA(cudaStreamSynchronize(s));
    }
    m.tc = Tree();
    SetKeys cen{m.cen_key.p, m.np}, qp{m.qp_key.p, m.nqp}, ch{m.chg_key.p, m.nc};
    // Point charges sit anywhere in their cells (on a corner, as the Born
    // ion's does), where a one-cell separation converges only like
    // (sqrt(3)/2)^p; when the products with the charges run as fast
    // multipole passes their tree interacts at two cells' separation
    // (ratio sqrt(3)/3): 5^3 neighbour leaves, offsets in [-5,5]^3.
    build_tree(m, m.tc, cen, qp, ch, charge_direct(m) ? 1 : 2);
}

void build_geometry_and_trees(Mesh &m, const double *d_panels, const double *d_charges) {
    cudaStream_t s = m.stream;
    const int TB = 256;
    const int64_t np = m.np, nq = m.nq, nqp = m.nqp;
    upload_rule((int)nq);

    // 1. geometry in the caller's order
    DArray<double> cen, nrm, area, qp, qw;
    cen.alloc(np * 3);
    nrm.alloc(np * 3);
    area.alloc(np);
    qp.alloc(nqp * 3);
    qw.alloc(nqp);
    DArray<int> bad;
    bad.alloc(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_panel_geometry<<<cdiv(np, TB), TB, 0, s>>>(d_panels, np, (int)nq, cen.p, nrm.p, area.p, qp.p,
                                                qw.p, bad.p);
    BEM_CHECK_LAUNCH();
    if (m.nc > 0) {
        k_check_charges<<<cdiv(m.nc, TB), TB, 0, s>>>(d_charges, m.nc, bad.p);
        BEM_CHECK_LAUNCH();
    }
    if (to_host(bad.p, s)) throw Error(BEM_EINVAL, "non-finite coordinate or zero-area panel");
    // optional: every charge must lie inside the (closed) surface
    if ((m.opt.flags & BEM_FLAG_CHECK_CHARGES) && m.nc > 0 && (double)m.nc * (double)np * 7.0 <= 4e10) {
        DArray<double> wind;
        wind.alloc(m.nc);
        BEM_CUDA(cudaMemsetAsync(wind.p, 0, m.nc * sizeof(double), s));
        const int64_t chunk = 4096;
        const int64_t nsplit = std::min<int64_t>(65535, (np + chunk - 1) / chunk);
        const int64_t ch = (np + nsplit - 1) / nsplit;
        k_winding<<<dim3(cdiv(m.nc, TB), (unsigned)nsplit), TB, 0, s>>>(d_panels, np, d_charges, m.nc, ch, wind.p);
        BEM_CHECK_LAUNCH();
        constexpr double kPi = 3.14159265358979323846;
        std::vector<double> w(m.nc);
        BEM_CUDA(cudaMemcpyAsync(w.data(), wind.p, m.nc * sizeof(double), cudaMemcpyDeviceToHost, s));
        BEM_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < m.nc; ++k)
            if (!(std::fabs(w[k] + 4.0 * kPi) < 2.0 * kPi))
                throw Error(BEM_EINVAL, "charge " + std::to_string(k) + " is not enclosed by the surface "
                                        "(winding " + std::to_string(w[k] / (4.0 * kPi)) + ")");
    }

    // 2. root cube: bounding cube of all vertices and charges, padded
    double lo[3], hi[3];
    compute_bbox(d_panels, np * 3, 3, lo, hi, s);
    if (m.nc > 0) {
        double lo2[3], hi2[3];
        compute_bbox(d_charges, m.nc, 4, lo2, hi2, s);
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], lo2[k]);
            hi[k] = std::max(hi[k], hi2[k]);
        }
    }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    if (!(ext > 0)) ext = 1.0;
    m.side = ext * (1.0 + 1e-6) + 1e-12;
    for (int k = 0; k < 3; ++k) m.root_min[k] = 0.5 * (lo[k] + hi[k]) - 0.5 * m.side;

    // 3. Morton keys and sort of centroids and quadrature points
    Root r = root_of(m);
    DArray<uint64_t> k0;
    DArray<int> i0;
    k0.alloc(std::max(np, nqp));
    i0.alloc(std::max(np, nqp));
    m.cen_key.alloc(np);
    m.cen_perm.alloc(np);
    k_keys<<<cdiv(np, TB), TB, 0, s>>>(cen.p, np, 3, r, k0.p, i0.p);
    BEM_CHECK_LAUNCH();
    sort_pairs(k0.p, i0.p, m.cen_key.p, m.cen_perm.p, np, s);
    DArray<int> qperm;
    qperm.alloc(nqp);
    m.qp_key.alloc(nqp);
    k_keys<<<cdiv(nqp, TB), TB, 0, s>>>(qp.p, nqp, 3, r, k0.p, i0.p);
    BEM_CHECK_LAUNCH();
    sort_pairs(k0.p, i0.p, m.qp_key.p, qperm.p, nqp, s);

    // 4. leaf level
    if (m.opt.depth > 0) {
        m.L = std::min(m.opt.depth, MORTON_BITS);
    } else if (m.opt.depth < 0) {
        m.L = 0;
    } else {
        DArray<unsigned long long> hist;
        hist.alloc(MORTON_BITS + 2);
        BEM_CUDA(cudaMemsetAsync(hist.p, 0, (MORTON_BITS + 2) * sizeof(unsigned long long), s));
        k_level_hist<<<std::min(1024, cdiv(np, 256)), 256, 0, s>>>(m.cen_key.p, np, hist.p);
        BEM_CHECK_LAUNCH();
        std::vector<unsigned long long> h(MORTON_BITS + 2);
        BEM_CUDA(cudaMemcpyAsync(h.data(), hist.p, h.size() * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
        BEM_CUDA(cudaStreamSynchronize(s));
        unsigned long long c = 1;
        m.L = MORTON_BITS;
        for (int l = 0; l <= MORTON_BITS; ++l) {
            c += h[l];
            if ((double)np / (double)c <= (double)m.opt.leaf_size) {
                m.L = l;
                break;
            }
        }
    }

    // 5. sorted panel data
    m.cen64.alloc(np * 3);
    m.nrm64.alloc(np * 3);
    m.area64.alloc(np);
    k_gather_rows<double><<<cdiv(np, TB), TB, 0, s>>>(cen.p, m.cen_perm.p, m.cen64.p, np, 3);
    k_gather_rows<double><<<cdiv(np, TB), TB, 0, s>>>(nrm.p, m.cen_perm.p, m.nrm64.p, np, 3);
    k_gather_rows<double><<<cdiv(np, TB), TB, 0, s>>>(area.p, m.cen_perm.p, m.area64.p, np, 1);
    BEM_CHECK_LAUNCH();
    DArray<int> rank;
    rank.alloc(np);
    k_inverse_perm<<<cdiv(np, TB), TB, 0, s>>>(m.cen_perm.p, rank.p, np);
    m.qp_panel.alloc(nqp);
    k_qp_panel<<<cdiv(nqp, TB), TB, 0, s>>>(qperm.p, rank.p, (int)nq, m.qp_panel.p, nqp);
    // each sorted panel's quadrature points in the rule's order, as sorted
    // positions: qp_of_panel[j nq + q] = inverse(qperm)[cen_perm[j] nq + q]
    {
        DArray<int> invq;
        invq.alloc(nqp);
        k_inverse_perm<<<cdiv(nqp, TB), TB, 0, s>>>(qperm.p, invq.p, nqp);
        m.qp_of_panel.alloc(nqp);
        k_qp_of_panel<<<cdiv(nqp, TB), TB, 0, s>>>(m.cen_perm.p, invq.p, (int)nq, np, m.qp_of_panel.p);
        BEM_CHECK_LAUNCH();
        BEM_CUDA(cudaStreamSynchronize(s));  // invq is released on return
    }
    m.qpg64.alloc(nqp * 3);
    m.qw64.alloc(nqp);
    k_gather_rows<double><<<cdiv(nqp, TB), TB, 0, s>>>(qp.p, qperm.p, m.qpg64.p, nqp, 3);
    k_gather_rows<double><<<cdiv(nqp, TB), TB, 0, s>>>(qw.p, qperm.p, m.qw64.p, nqp, 1);
    BEM_CHECK_LAUNCH();
    LeafGeom g = leaf_geom(m);
    if (m.opt.precision == BEM_MIXED) {
        m.cen32.alloc(np);
        m.nrm32.alloc(np);
        m.qp32.alloc(nqp);
    } else {
        m.cen64r.alloc(np);
        m.nrm64r.alloc(np);
        m.qp64r.alloc(nqp);
    }
    k_rel_records<<<cdiv(np, TB), TB, 0, s>>>(m.cen64.p, nullptr, m.nrm64.p, m.cen_key.p, np, g,
                                              m.cen32.p, m.cen64r.p, m.nrm32.p, m.nrm64r.p);
    k_rel_records<<<cdiv(nqp, TB), TB, 0, s>>>(m.qpg64.p, m.qw64.p, nullptr, m.qp_key.p, nqp, g,
                                               m.qp32.p, m.qp64r.p, nullptr, nullptr);
    BEM_CHECK_LAUNCH();

    // 6. trees
    SetKeys sc{m.cen_key.p, np}, sq{m.qp_key.p, nqp}, none{};
    build_tree(m, m.tp, sc, sq, none, 1);
    build_charges(m, d_charges);
    BEM_CUDA(cudaStreamSynchronize(s));
}

void rebuild_charge_tree(Mesh &m, const double *d_charges) { build_charges(m, d_charges); }

void exclusive_scan_int(const int *in, int *out, int n, cudaStream_t s) { scan_exclusive(in, out, n, s); }

}  // namespace bem
