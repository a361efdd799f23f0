// Higher-accuracy integration of the charge-panel pairs (Sec. 2.1 names the
// exact integrals over flat panels as the alternative to quadrature).
//
// With BEM_FLAG_CHARGE_NEAR_EXACT, every pair of a charge x_k and a panel j
// whose centroid lies within 2.5 sqrt(A_j) of x_k takes the exact
// single-layer integral over the flat panel instead of the quadrature rule in
// C s (the potential of the surface charge at the charges, Eq. reac), in
// C^T q and in grad_x (C s).  The products themselves keep the rule (direct
// sums or fast multipole passes); a table of FP64 corrections
//   E_kj = [int_Tj dA / |x_k - y| - sum_q A_j w_q / |x_k - y_jq|] / (4 pi)
// and of their gradients in x_k is added afterwards, by charge for C s and
// grad C s, by panel (the table's transpose) for C^T q.  The pairs are found
// through the charge tree's neighbour lists, which reach every such panel
// when 2.5 sqrt(A_max) is at most the tree's separation in cells times the
// leaf width (checked; otherwise every panel is tried when n_c n_p <= 2e9).
#include <cmath>
#include <cstring>

#include "bem_internal.cuh"

namespace bem {

namespace {

// 4 pi times the single-layer potential of a unit density on the flat
// triangle v[9] at t, and 4 pi times its gradient.  With a_k = v_k - t, the
// unit normal nu, the height h = (t - v_0).nu of t and the solid angle Om
// the triangle subtends at t (positive on the side of nu; the triple-product
// formula), the divergence theorem in the triangle's plane gives
//   int_T dA / R = sum_e d_e L_e - h Om,
//   int_T (t - y) / R^3 dA = nu Om + sum_e m_e L_e,
// with m_e the outward in-plane normal of edge e, d_e = m_e.a_e the distance
// of t's foot from the edge's line and L_e = int_e dl / R (one logarithm).
__device__ void tri_single_layer_4pi(const double t[3], const double *v, double &S, double g[3]) {
    double a[3][3];
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) a[k][c] = v[3 * k + c] - t[c];
    auto dot = [](const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    const double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
    const double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    double nu[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double lnu = sqrt(dot(nu, nu));
    for (int c = 0; c < 3; ++c) nu[c] /= lnu;
    double len[3];
    for (int k = 0; k < 3; ++k) len[k] = sqrt(dot(a[k], a[k]));
    const double c12[3] = {a[1][1] * a[2][2] - a[1][2] * a[2][1], a[1][2] * a[2][0] - a[1][0] * a[2][2],
                           a[1][0] * a[2][1] - a[1][1] * a[2][0]};
    const double den = len[0] * len[1] * len[2] + dot(a[0], a[1]) * len[2] + dot(a[0], a[2]) * len[1] +
                       dot(a[1], a[2]) * len[0];
    // atan2 gives half the angle seen with the vertices counter-clockwise,
    // i.e. from the side opposite to nu
    const double om = -2.0 * atan2(dot(a[0], c12), den);
    const double h = -dot(a[0], nu);
    S = -h * om;
    double f[3] = {nu[0] * om, nu[1] * om, nu[2] * om};
    for (int e = 0; e < 3; ++e) {
        const int b = (e + 1) % 3;
        double te[3] = {a[b][0] - a[e][0], a[b][1] - a[e][1], a[b][2] - a[e][2]};
        const double lt = sqrt(dot(te, te));
        for (int c = 0; c < 3; ++c) te[c] /= lt;
        const double m[3] = {te[1] * nu[2] - te[2] * nu[1], te[2] * nu[0] - te[0] * nu[2],
                             te[0] * nu[1] - te[1] * nu[0]};
        const double sa = dot(a[e], te), sb = dot(a[b], te);
        // the two algebraically equal forms; the one without cancellation
        const double lg = (sa + sb >= 0.0) ? log((len[b] + sb) / (len[e] + sa)) : log((len[e] - sa) / (len[b] - sb));
        const double d = dot(m, a[e]);
        if (d != 0.0) S += d * lg;
        for (int c = 0; c < 3; ++c) f[c] += m[c] * lg;
    }
    for (int c = 0; c < 3; ++c) g[c] = -f[c];
}

// the largest panel area (non-negative doubles order like their bit patterns)
__global__ void k_amax(const double *a, int64_t n, unsigned long long *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) v = (unsigned long long)__double_as_longlong(a[i]);
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(out, v);
}

__global__ void k_leaf_of_chg(const int *beg, int *leaf_of) {
    const int l = blockIdx.x;
    for (int i = beg[l] + threadIdx.x; i < beg[l + 1]; i += blockDim.x) leaf_of[i] = l;
}

// Pairs of charge k (sorted order): the panels j of the leaves adjacent to
// k's leaf with |x_k - c_j|^2 <= 6.25 A_j.  Writes the count (cnt) or, with
// off set, the panels of k's entries in increasing order.
__global__ void k_cnear_pairs(int64_t nc, const int *leaf_of, const int *nbr_off, const int *nbr,
                              const int *cen_beg, const double *xq, const double *cen, const double *area,
                              const int *off, int *cnt, int *col) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const double x[3] = {xq[3 * k], xq[3 * k + 1], xq[3 * k + 2]};
    const int L = leaf_of[k];
    int n = 0;
    const int base = off ? off[k] : 0;
    for (int e = nbr_off[L]; e < nbr_off[L + 1]; ++e) {
        const int S = nbr[e];
        for (int j = cen_beg[S]; j < cen_beg[S + 1]; ++j) {
            const double dx = x[0] - cen[3 * j], dy = x[1] - cen[3 * j + 1], dz = x[2] - cen[3 * j + 2];
            if (dx * dx + dy * dy + dz * dz > 6.25 * area[j]) continue;
            if (off) col[base + n] = j;
            ++n;
        }
    }
    if (!off) cnt[k] = n;
}

// the same over every panel (when the neighbour lists do not reach far
// enough and n_c x n_p is small)
__global__ void k_cnear_pairs_all(int64_t nc, int64_t np, const double *xq, const double *cen, const double *area,
                                  const int *off, int *cnt, int *col) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const double x[3] = {xq[3 * k], xq[3 * k + 1], xq[3 * k + 2]};
    int n = 0;
    const int base = off ? off[k] : 0;
    for (int64_t j = 0; j < np; ++j) {
        const double dx = x[0] - cen[3 * j], dy = x[1] - cen[3 * j + 1], dz = x[2] - cen[3 * j + 2];
        if (dx * dx + dy * dy + dz * dz > 6.25 * area[j]) continue;
        if (off) col[base + n] = (int)j;
        ++n;
    }
    if (!off) cnt[k] = n;
}

// the panels of each charge's row in increasing order (a handful per row)
__global__ void k_cnear_sort_rows(const int *off, int64_t nc, int *col) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    for (int a = off[k] + 1; a < off[k + 1]; ++a) {
        const int v = col[a];
        int b = a - 1;
        while (b >= off[k] && col[b] > v) {
            col[b + 1] = col[b];
            --b;
        }
        col[b + 1] = v;
    }
}

__global__ void k_cnear_rows(const int *off, int64_t nc, int *row) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    for (int e = off[k]; e < off[k + 1]; ++e) row[e] = (int)k;
}

// entry e = (charge row[e], panel col[e]): (exact - rule) / (4 pi) of the
// potential and of its gradient in x_k, in FP64
__global__ void k_cnear_values(int64_t nnz, const int *row, const int *col, const double *xq, const double *pan,
                               const double *qpg, const double *qw, const int *qp_of_panel, int nq,
                               double *val) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int k = row[e], j = col[e];
    const double x[3] = {xq[3 * k], xq[3 * k + 1], xq[3 * k + 2]};
    double S, g[3];
    tri_single_layer_4pi(x, pan + 9 * (int64_t)j, S, g);
    for (int q = 0; q < nq; ++q) {
        const int i = qp_of_panel[(int64_t)j * nq + q];
        const double d[3] = {x[0] - qpg[3 * i], x[1] - qpg[3 * i + 1], x[2] - qpg[3 * i + 2]};
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
        S -= qw[i] / r;
        const double f = qw[i] / (r2 * r);  // minus the rule's gradient term -w d / r^3
        for (int c = 0; c < 3; ++c) g[c] += f * d[c];
    }
    val[4 * e] = S / FOUR_PI;
    for (int c = 0; c < 3; ++c) val[4 * e + 1 + c] = g[c] / FOUR_PI;
}

__global__ void k_iota_entries(int64_t n, int *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) out[e] = (int)e;
}

// panel vertices in the sorted panel order (perm: sorted -> caller's index)
__global__ void k_gather_panels(const double *pan, const int *perm, int64_t np, double *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np * 9) return;
    const int64_t j = i / 9;
    out[i] = pan[9 * (int64_t)perm[j] + (i - 9 * j)];
}

__global__ void k_count_cols(const int *col, int64_t nnz, int *cnt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(cnt + col[e], 1);
}

// the transpose's entries in the order of the stable sort by panel (within
// a panel, increasing charge)
__global__ void k_cnear_transpose(const int *perm, const int *row, const double *val, int64_t nnz, int *trow,
                                  double *tval) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const int e = perm[p];
    trow[p] = row[e];
    tval[p] = val[4 * e];
}

// out[k * stride + c] += sum_e val[4 e + c] s[col[e]], c < ncomp
__global__ void k_cnear_apply(const int *off, const int *col, const double *val, const double *s, int64_t nc,
                              int stride, int ncomp, double *out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nc) return;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = off[k]; e < off[k + 1]; ++e) {
        const double sj = s[col[e]];
        for (int c = 0; c < ncomp; ++c) a[c] = fma(val[4 * e + c], sj, a[c]);
    }
    for (int c = 0; c < ncomp; ++c) out[k * stride + c] += a[c];
}

// v[j] += sum over the charges k of panel j's entries of E_kj u[k]
__global__ void k_cnear_apply_t(const int *toff, const int *trow, const double *tval, const double *u, int64_t np,
                                double *v) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double a = 0.0;
    for (int e = toff[j]; e < toff[j + 1]; ++e) a = fma(tval[e], u[trow[e]], a);
    v[j] += a;
}

}  // namespace

bool charge_near_on(const Mesh &m) { return (m.opt.flags & BEM_FLAG_CHARGE_NEAR_EXACT) && m.nc > 0; }

void keep_panel_vertices(Mesh &m, const double *d_panels) {
    if (!(m.opt.flags & BEM_FLAG_CHARGE_NEAR_EXACT)) return;
    m.pan64.alloc((size_t)m.np * 9);
    k_gather_panels<<<cdiv(m.np * 9, 256), 256, 0, m.stream>>>(d_panels, m.cen_perm.p, m.np, m.pan64.p);
    BEM_CHECK_LAUNCH();
}

void build_charge_near(Mesh &m) {
    m.cn_nnz = 0;
    if (!charge_near_on(m)) return;
    if (m.pan64.n < (size_t)m.np * 9) throw Error(BEM_ECUDA, "charge-panel pairs: panel vertices not kept");
    cudaStream_t s = m.stream;
    const Tree &t = m.tc;
    const int64_t nc = m.nc, np = m.np;
    // the neighbour lists must reach every panel within 2.5 sqrt(A_max)
    DArray<unsigned long long> amax;
    amax.alloc(1);
    BEM_CUDA(cudaMemsetAsync(amax.p, 0, sizeof(unsigned long long), s));
    k_amax<<<cdiv(np, 256), 256, 0, s>>>(m.area64.p, np, amax.p);
    BEM_CHECK_LAUNCH();
    unsigned long long bits = 0;
    BEM_CUDA(cudaMemcpyAsync(&bits, amax.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    double a_max = 0.0;
    std::memcpy(&a_max, &bits, sizeof(a_max));
    const double leaf_w = m.side / (double)(1 << t.L);
    const bool reach = t.L == 0 || 2.5 * std::sqrt(a_max) <= t.ws * leaf_w;
    if (!reach && (double)nc * (double)np > 2e9)
        throw Error(BEM_EUNSUPPORTED, "charge-panel pairs: panels larger than the charge tree's neighbour reach");
    auto pairs = [&](const int *off, int *cnt, int *col, const int *leaf_of) {
        if (reach)
            k_cnear_pairs<<<cdiv(nc, 128), 128, 0, s>>>(nc, leaf_of, t.nbr_off.p, t.nbr.p, t.cen_beg.p, m.chgg64.p,
                                                        m.cen64.p, m.area64.p, off, cnt, col);
        else
            k_cnear_pairs_all<<<cdiv(nc, 128), 128, 0, s>>>(nc, np, m.chgg64.p, m.cen64.p, m.area64.p, off, cnt, col);
        BEM_CHECK_LAUNCH();
    };
    DArray<int> leaf_of, cnt, row, perm0, perm, keys;
    leaf_of.alloc(nc);
    k_leaf_of_chg<<<t.nleaf, 128, 0, s>>>(t.chg_beg.p, leaf_of.p);
    BEM_CHECK_LAUNCH();
    cnt.alloc(nc + 1);
    BEM_CUDA(cudaMemsetAsync(cnt.p, 0, (nc + 1) * sizeof(int), s));
    pairs(nullptr, cnt.p, nullptr, leaf_of.p);
    m.cn_off.alloc(nc + 1);
    scan_exclusive_i32(cnt.p, m.cn_off.p, nc + 1, s);
    int nnz = 0;
    BEM_CUDA(cudaMemcpyAsync(&nnz, m.cn_off.p + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
    BEM_CUDA(cudaStreamSynchronize(s));
    m.cn_nnz = nnz;
    m.cn_col.alloc(nnz);
    m.cn_val.alloc((size_t)nnz * 4);
    m.cnT_off.alloc(np + 1);
    m.cnT_row.alloc(nnz);
    m.cnT_val.alloc(nnz);
    if (nnz == 0) return;
    pairs(m.cn_off.p, nullptr, m.cn_col.p, leaf_of.p);
    k_cnear_sort_rows<<<cdiv(nc, 128), 128, 0, s>>>(m.cn_off.p, nc, m.cn_col.p);
    row.alloc(nnz);
    k_cnear_rows<<<cdiv(nc, 128), 128, 0, s>>>(m.cn_off.p, nc, row.p);
    BEM_CHECK_LAUNCH();
    k_cnear_values<<<cdiv(nnz, 128), 128, 0, s>>>(nnz, row.p, m.cn_col.p, m.chgg64.p, m.pan64.p, m.qpg64.p,
                                                  m.qw64.p, m.qp_of_panel.p, (int)m.nq, m.cn_val.p);
    BEM_CHECK_LAUNCH();
    // the transpose: entries stably sorted by panel, offsets from the counts
    int bits_np = 1;
    while (((int64_t)1 << bits_np) < np) ++bits_np;
    perm0.alloc(nnz);
    perm.alloc(nnz);
    keys.alloc(nnz);
    k_iota_entries<<<cdiv(nnz, 256), 256, 0, s>>>(nnz, perm0.p);
    BEM_CHECK_LAUNCH();
    sort_pairs_int(m.cn_col.p, perm0.p, keys.p, perm.p, nnz, bits_np, s);
    cnt.alloc(np + 1);
    BEM_CUDA(cudaMemsetAsync(cnt.p, 0, (np + 1) * sizeof(int), s));
    k_count_cols<<<cdiv(nnz, 256), 256, 0, s>>>(m.cn_col.p, nnz, cnt.p);
    BEM_CHECK_LAUNCH();
    scan_exclusive_i32(cnt.p, m.cnT_off.p, np + 1, s);
    k_cnear_transpose<<<cdiv(nnz, 256), 256, 0, s>>>(perm.p, row.p, m.cn_val.p, nnz, m.cnT_row.p, m.cnT_val.p);
    BEM_CHECK_LAUNCH();
    BEM_CUDA(cudaStreamSynchronize(s));  // the temporaries are released on return
}

void charge_near_phi(Mesh &m, const double *s_sorted, double *out, int stride, int ncomp) {
    if (!charge_near_on(m) || m.cn_nnz == 0) return;
    k_cnear_apply<<<cdiv(m.nc, 128), 128, 0, m.stream>>>(m.cn_off.p, m.cn_col.p, m.cn_val.p, s_sorted, m.nc, stride,
                                                         ncomp, out);
    BEM_CHECK_LAUNCH();
}

void charge_near_ct(Mesh &m, const double *u_sorted, double *v) {
    if (!charge_near_on(m) || m.cn_nnz == 0) return;
    k_cnear_apply_t<<<cdiv(m.np, 256), 256, 0, m.stream>>>(m.cnT_off.p, m.cnT_row.p, m.cnT_val.p, u_sorted, m.np,
                                                           v);
    BEM_CHECK_LAUNCH();
}

}  // namespace bem
