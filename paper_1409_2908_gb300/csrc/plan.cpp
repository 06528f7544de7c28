// Host plan layer: exact validation of a base case against the Brent
// equations (Eq. 2), unrolling of L recursive steps into R^L leaf products
// with their operand and output block lists (Section 3.1 applied
// recursively), normalisation of the coefficient chains (Section 3.1: scalar
// factors are piped through to the leaf call), and upload to the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>

#include "fmm_internal.h"

namespace fmm {

namespace {

// x = mant * 2^exp exactly, mant odd (or 0).
void dyadic(double x, int64_t *mant, int *exp) {
    if (x == 0.0) {
        *mant = 0;
        *exp = 0;
        return;
    }
    int e;
    double f = std::frexp(x, &e);              // x = f * 2^e, |f| in [0.5, 1)
    int64_t m = (int64_t)std::ldexp(f, 53);    // exact: 53-bit significand
    e -= 53;
    while ((m & 1) == 0) {
        m /= 2;
        ++e;
    }
    *mant = m;
    *exp = e;
}

// Scale a matrix of doubles to integers: x = G * 2^emin exactly.
bool to_integers(const double *X, size_t n, std::vector<__int128> *G, int *emin) {
    int lo = 1 << 30;
    std::vector<int64_t> m(n);
    std::vector<int> e(n);
    for (size_t i = 0; i < n; ++i) {
        if (!std::isfinite(X[i])) return false;
        dyadic(X[i], &m[i], &e[i]);
        if (m[i] != 0) lo = std::min(lo, e[i]);
    }
    if (lo == (1 << 30)) lo = 0;
    G->assign(n, 0);
    for (size_t i = 0; i < n; ++i) {
        if (m[i] == 0) continue;
        int sh = e[i] - lo;
        int bits = 64 - __builtin_clzll((unsigned long long)std::llabs(m[i]));
        if (sh + bits > 40) return false;      // keep products in range
        (*G)[i] = (__int128)m[i] << sh;
    }
    *emin = lo;
    return true;
}

}  // namespace

// Eq. (2): sum_r U_ir V_jr W_qr equals the <M,K,N> matmul tensor, where
// T_ijq = 1 exactly when i = a*K + b, j = b*N + c, q = a*N + c.
bool brent_exact(int M, int K, int N, int R, const double *U, const double *V,
                 const double *W, bool *representable) {
    const int I = M * K, J = K * N, Q = M * N;
    std::vector<__int128> gu, gv, gw;
    int eu, ev, ew;
    *representable = to_integers(U, (size_t)I * R, &gu, &eu) &&
                     to_integers(V, (size_t)J * R, &gv, &ev) &&
                     to_integers(W, (size_t)Q * R, &gw, &ew);
    if (!*representable) return false;
    const int E = eu + ev + ew;                  // real sum = S * 2^E
    std::vector<__int128> S((size_t)I * J * Q, 0);
    for (int r = 0; r < R; ++r)
        for (int i = 0; i < I; ++i) {
            if (gu[(size_t)i * R + r] == 0) continue;
            for (int j = 0; j < J; ++j) {
                if (gv[(size_t)j * R + r] == 0) continue;
                const __int128 uv = gu[(size_t)i * R + r] * gv[(size_t)j * R + r];
                for (int q = 0; q < Q; ++q)
                    if (gw[(size_t)q * R + r] != 0)
                        S[((size_t)i * J + j) * Q + q] += uv * gw[(size_t)q * R + r];
            }
        }
    __int128 one;                                // 2^-E as an integer
    if (E > 0) {
        one = -1;                                // a sum of 1 is impossible
    } else {
        if (-E > 120) return false;
        one = (__int128)1 << (-E);
    }
    for (int i = 0; i < I; ++i)
        for (int j = 0; j < J; ++j)
            for (int q = 0; q < Q; ++q) {
                const int a = i / K, b = i % K;
                const bool t = (j / N == b) && (q / N == a) && (q % N == j % N);
                const __int128 s = S[((size_t)i * J + j) * Q + q];
                if (t ? (s != one) : (s != 0)) return false;
            }
    return true;
}

// Unroll L steps: leaf r = (r_1..r_L); block (i_1..i_L), i_l = x_l*Q + y_l
// of a P x Q split, sits at row sum x_l P^(L-l), col sum y_l Q^(L-l).
static void unroll(const double *F, int P, int Q, int R, int L, TermList *out) {
    const int PQ = P * Q;
    std::vector<std::vector<int>> nz(R);
    for (int r = 0; r < R; ++r)
        for (int i = 0; i < PQ; ++i)
            if (F[(size_t)i * R + r] != 0.0) nz[r].push_back(i);
    int64_t leaves = 1;
    for (int l = 0; l < L; ++l) leaves *= R;
    out->ptr.assign(leaves + 1, 0);
    out->row.clear();
    out->col.clear();
    out->coef.clear();
    std::vector<int> digit(L);
    struct T { int32_t row, col; double coef; };
    std::vector<T> buf;
    for (int64_t leaf = 0; leaf < leaves; ++leaf) {
        int64_t x = leaf;
        for (int l = L - 1; l >= 0; --l) {
            digit[l] = int(x % R);
            x /= R;
        }
        buf.clear();
        // odometer over the nonzeros of each level's column
        std::vector<size_t> pos(L, 0);
        bool empty = false;
        for (int l = 0; l < L; ++l)
            if (nz[digit[l]].empty()) empty = true;
        while (!empty) {
            int32_t row = 0, col = 0;
            double coef = 1.0;
            for (int l = 0; l < L; ++l) {
                const int i = nz[digit[l]][pos[l]];
                row = row * P + i / Q;
                col = col * Q + i % Q;
                coef *= F[(size_t)i * R + digit[l]];
            }
            buf.push_back({row, col, coef});
            int l = L - 1;
            while (l >= 0) {
                if (++pos[l] < nz[digit[l]].size()) break;
                pos[l] = 0;
                --l;
            }
            if (l < 0) break;
        }
        std::sort(buf.begin(), buf.end(), [](const T &u, const T &v) {
            return u.row != v.row ? u.row < v.row : u.col < v.col;
        });
        for (const T &t : buf) {
            out->row.push_back(t.row);
            out->col.push_back(t.col);
            out->coef.push_back(t.coef);
        }
        out->ptr[leaf + 1] = (int64_t)out->row.size();
    }
}

// Divide a leaf's chain by its first coefficient when every ratio is exact;
// returns the scale taken out (1 when the chain is left as it is).
static double normalise_chain(const double *c, int64_t n, double *out) {
    const double s = c[0];
    bool exact = true;
    for (int64_t t = 0; t < n && exact; ++t) {
        const double q = c[t] / s;
        if (q * s != c[t]) exact = false;
    }
    if (!exact) {
        for (int64_t t = 0; t < n; ++t) out[t] = c[t];
        return 1.0;
    }
    for (int64_t t = 0; t < n; ++t) out[t] = c[t] / s;
    return s;
}

fmm_status build_plan(fmm_plan *p, int M, int K, int N, int R, const double *U,
                      const double *V, const double *W, int L) {
    p->M = M; p->K = K; p->N = N; p->R = R; p->L = L;
    int64_t leaves = 1;
    for (int l = 0; l < L; ++l) {
        leaves *= R;
        if (leaves > (int64_t(1) << 20)) return FMM_ERR_UNSUPPORTED;
    }
    int64_t side = 1;
    for (int l = 0; l < L; ++l) {
        side *= std::max(M, std::max(K, N));
        if (side > 32768) return FMM_ERR_UNSUPPORTED;
    }
    p->leaves = leaves;
    p->U.assign(U, U + (size_t)M * K * R);
    p->V.assign(V, V + (size_t)K * N * R);
    p->W.assign(W, W + (size_t)M * N * R);
    p->integer_coefs = true;
    for (const std::vector<double> *F : {&p->U, &p->V, &p->W})
        for (double c : *F)
            if (c != std::floor(c) || std::fabs(c) > 127.0) p->integer_coefs = false;
    unroll(U, M, K, R, L, &p->a);
    unroll(V, K, N, R, L, &p->b);
    unroll(W, M, N, R, L, &p->c);
    const int64_t cap = int64_t(1) << 25;
    if ((int64_t)p->a.row.size() > cap || (int64_t)p->b.row.size() > cap ||
        (int64_t)p->c.row.size() > cap)
        return FMM_ERR_UNSUPPORTED;
    p->a_norm.resize(p->a.coef.size());
    p->b_norm.resize(p->b.coef.size());
    p->c_scaled.resize(p->c.coef.size());
    p->slot_of_leaf_a.assign(leaves, -1);
    p->slot_of_leaf_b.assign(leaves, -1);
    p->slots_a = p->slots_b = 0;
    for (int64_t r = 0; r < leaves; ++r) {
        const int64_t a0 = p->a.ptr[r], a1 = p->a.ptr[r + 1];
        const int64_t b0 = p->b.ptr[r], b1 = p->b.ptr[r + 1];
        double sA = 1.0, sB = 1.0;
        if (a1 > a0) sA = normalise_chain(&p->a.coef[a0], a1 - a0, &p->a_norm[a0]);
        if (b1 > b0) sB = normalise_chain(&p->b.coef[b0], b1 - b0, &p->b_norm[b0]);
        for (int64_t t = p->c.ptr[r]; t < p->c.ptr[r + 1]; ++t)
            p->c_scaled[t] = p->c.coef[t] * sA * sB;
        if (a1 - a0 > 1) p->slot_of_leaf_a[r] = int32_t(p->slots_a++);
        if (b1 - b0 > 1) p->slot_of_leaf_b[r] = int32_t(p->slots_b++);
    }
    return FMM_OK;
}

namespace {
struct Blob {
    size_t bytes = 0;
    template <class T> size_t add(size_t n) {
        size_t off = (bytes + 255) & ~size_t(255);
        bytes = off + n * sizeof(T);
        return off;
    }
};
}  // namespace

fmm_status upload_plan(fmm_plan *p) {
    const int64_t leaves = p->leaves;
    const int64_t na = p->a.row.size(), nb = p->b.row.size(), nc = p->c.row.size();
    int64_t side_m = 1, side_n = 1;
    for (int l = 0; l < p->L; ++l) { side_m *= p->M; side_n *= p->N; }
    const int64_t cblocks = side_m * side_n;

    // host images
    std::vector<int> a_ptr(leaves + 1), b_ptr(leaves + 1), c_ptr(leaves + 1);
    std::vector<int> a_code(na), b_code(nb), c_code(nc);
    for (int64_t r = 0; r <= leaves; ++r) {
        a_ptr[r] = int(p->a.ptr[r]);
        b_ptr[r] = int(p->b.ptr[r]);
        c_ptr[r] = int(p->c.ptr[r]);
    }
    for (int64_t t = 0; t < na; ++t) a_code[t] = (p->a.row[t] << 16) | p->a.col[t];
    for (int64_t t = 0; t < nb; ++t) b_code[t] = (p->b.row[t] << 16) | p->b.col[t];
    for (int64_t t = 0; t < nc; ++t) c_code[t] = (p->c.row[t] << 16) | p->c.col[t];
    std::vector<int> ua_code(leaves), ub_code(leaves), u_ptr(leaves + 1);
    std::vector<double> u_one(leaves, 1.0);
    std::vector<int> sa_leaf(std::max<int64_t>(p->slots_a, 1)), sb_leaf(std::max<int64_t>(p->slots_b, 1));
    for (int64_t r = 0; r < leaves; ++r) {
        u_ptr[r] = int(r);
        const int sa = p->slot_of_leaf_a[r], sb = p->slot_of_leaf_b[r];
        if (sa >= 0) { ua_code[r] = -(sa + 1); sa_leaf[sa] = int(r); }
        else ua_code[r] = p->a.ptr[r + 1] > p->a.ptr[r] ? a_code[p->a.ptr[r]] : 0;
        if (sb >= 0) { ub_code[r] = -(sb + 1); sb_leaf[sb] = int(r); }
        else ub_code[r] = p->b.ptr[r + 1] > p->b.ptr[r] ? b_code[p->b.ptr[r]] : 0;
    }
    u_ptr[leaves] = int(leaves);
    // transpose of the C lists: per C block, (leaf, coefficient) by leaf
    std::vector<int> cq_ptr(cblocks + 1, 0), cq_leaf(nc);
    std::vector<double> cq_coef(nc);
    for (int64_t t = 0; t < nc; ++t) cq_ptr[(int64_t)p->c.row[t] * side_n + p->c.col[t] + 1]++;
    for (int64_t q = 0; q < cblocks; ++q) cq_ptr[q + 1] += cq_ptr[q];
    {
        std::vector<int> fill(cq_ptr.begin(), cq_ptr.end() - 1);
        for (int64_t r = 0; r < leaves; ++r)
            for (int64_t t = p->c.ptr[r]; t < p->c.ptr[r + 1]; ++t) {
                const int64_t q = (int64_t)p->c.row[t] * side_n + p->c.col[t];
                const bool live = p->a.ptr[r + 1] > p->a.ptr[r] && p->b.ptr[r + 1] > p->b.ptr[r];
                cq_leaf[fill[q]] = int(r);
                cq_coef[fill[q]] = live ? p->c_scaled[t] : 0.0;
                fill[q]++;
            }
    }
    std::vector<double> c_coef_dev(p->c_scaled);
    // leaves whose A or B chain is empty would read nothing; give them an
    // empty epilogue by zeroing their coefficients
    for (int64_t r = 0; r < leaves; ++r) {
        const bool live = p->a.ptr[r + 1] > p->a.ptr[r] && p->b.ptr[r + 1] > p->b.ptr[r];
        if (!live)
            for (int64_t t = p->c.ptr[r]; t < p->c.ptr[r + 1]; ++t) c_coef_dev[t] = 0.0;
    }

    // level-by-level scheme: base lists of U and V by column, W by row
    const int R = p->R, MK = p->M * p->K, KN = p->K * p->N, MN = p->M * p->N;
    std::vector<int> lu_ptr(R + 1, 0), lv_ptr(R + 1, 0), lw_ptr(MN + 1, 0), lu_code, lv_code, lw_r;
    std::vector<double> lu_coef, lv_coef, lw_coef;
    for (int r = 0; r < R; ++r) {
        for (int i = 0; i < MK; ++i)
            if (p->U[(size_t)i * R + r] != 0.0) {
                lu_code.push_back(((i / p->K) << 16) | (i % p->K));
                lu_coef.push_back(p->U[(size_t)i * R + r]);
            }
        lu_ptr[r + 1] = int(lu_code.size());
        for (int j = 0; j < KN; ++j)
            if (p->V[(size_t)j * R + r] != 0.0) {
                lv_code.push_back(((j / p->N) << 16) | (j % p->N));
                lv_coef.push_back(p->V[(size_t)j * R + r]);
            }
        lv_ptr[r + 1] = int(lv_code.size());
    }
    for (int q = 0; q < MN; ++q) {
        for (int r = 0; r < R; ++r)
            if (p->W[(size_t)q * R + r] != 0.0) {
                lw_r.push_back(r);
                lw_coef.push_back(p->W[(size_t)q * R + r]);
            }
        lw_ptr[q + 1] = int(lw_r.size());
    }
    // integer copies of the base coefficients (residue-space recursion)
    auto to_int = [&](const std::vector<double> &v, std::vector<int> *out) {
        out->resize(v.size() + 1, 0);
        for (size_t i = 0; i < v.size(); ++i) {
            const double c = v[i];
            (*out)[i] = (c == std::floor(c) && std::fabs(c) <= 127.0) ? int(c) : 0;
        }
    };
    std::vector<int> lu_icoef, lv_icoef, lw_icoef;
    std::vector<int> lvt_code(lv_code.size() + 1, 0);
    for (size_t t = 0; t < lv_code.size(); ++t)
        lvt_code[t] = ((lv_code[t] & 0xffff) << 16) | (lv_code[t] >> 16);
    to_int(lu_coef, &lu_icoef);
    to_int(lv_coef, &lv_icoef);
    to_int(lw_coef, &lw_icoef);
    std::vector<int> leaf_slot(leaves);
    for (int64_t r = 0; r < leaves; ++r) leaf_slot[r] = -int(r + 1);
    std::vector<double> c_coef_raw(p->c.coef);
    for (int64_t r = 0; r < leaves; ++r) {
        const bool live = p->a.ptr[r + 1] > p->a.ptr[r] && p->b.ptr[r + 1] > p->b.ptr[r];
        if (!live)
            for (int64_t t = p->c.ptr[r]; t < p->c.ptr[r + 1]; ++t) c_coef_raw[t] = 0.0;
    }

    Blob bl;
    const size_t o_a_ptr = bl.add<int>(leaves + 1), o_a_code = bl.add<int>(na), o_a_coef = bl.add<double>(na);
    const size_t o_b_ptr = bl.add<int>(leaves + 1), o_b_code = bl.add<int>(nb), o_b_coef = bl.add<double>(nb);
    const size_t o_c_ptr = bl.add<int>(leaves + 1), o_c_code = bl.add<int>(nc), o_c_coef = bl.add<double>(nc);
    const size_t o_ua = bl.add<int>(leaves), o_ub = bl.add<int>(leaves), o_uptr = bl.add<int>(leaves + 1);
    const size_t o_one = bl.add<double>(leaves);
    const size_t o_sa = bl.add<int>(sa_leaf.size()), o_sb = bl.add<int>(sb_leaf.size());
    const size_t o_cq_ptr = bl.add<int>(cblocks + 1), o_cq_leaf = bl.add<int>(nc), o_cq_coef = bl.add<double>(nc);
    const size_t o_lu_ptr = bl.add<int>(R + 1), o_lu_code = bl.add<int>(lu_code.size() + 1),
                 o_lu_coef = bl.add<double>(lu_coef.size() + 1);
    const size_t o_lv_ptr = bl.add<int>(R + 1), o_lv_code = bl.add<int>(lv_code.size() + 1),
                 o_lv_coef = bl.add<double>(lv_coef.size() + 1);
    const size_t o_lw_ptr = bl.add<int>(MN + 1), o_lw_r = bl.add<int>(lw_r.size() + 1),
                 o_lw_coef = bl.add<double>(lw_coef.size() + 1);
    const size_t o_leaf_slot = bl.add<int>(leaves), o_c_raw = bl.add<double>(nc);
    const size_t o_a_raw = bl.add<double>(na), o_b_raw = bl.add<double>(nb);
    const size_t o_lu_i = bl.add<int>(lu_icoef.size()), o_lv_i = bl.add<int>(lv_icoef.size()),
                 o_lw_i = bl.add<int>(lw_icoef.size()), o_lvt = bl.add<int>(lvt_code.size());

    std::vector<unsigned char> host(bl.bytes, 0);
    auto put = [&](size_t off, const void *src, size_t n) { if (n) std::memcpy(host.data() + off, src, n); };
    put(o_a_ptr, a_ptr.data(), a_ptr.size() * 4);
    put(o_a_code, a_code.data(), a_code.size() * 4);
    put(o_a_coef, p->a_norm.data(), p->a_norm.size() * 8);
    put(o_b_ptr, b_ptr.data(), b_ptr.size() * 4);
    put(o_b_code, b_code.data(), b_code.size() * 4);
    put(o_b_coef, p->b_norm.data(), p->b_norm.size() * 8);
    put(o_c_ptr, c_ptr.data(), c_ptr.size() * 4);
    put(o_c_code, c_code.data(), c_code.size() * 4);
    put(o_c_coef, c_coef_dev.data(), c_coef_dev.size() * 8);
    put(o_ua, ua_code.data(), ua_code.size() * 4);
    put(o_ub, ub_code.data(), ub_code.size() * 4);
    put(o_uptr, u_ptr.data(), u_ptr.size() * 4);
    put(o_one, u_one.data(), u_one.size() * 8);
    put(o_sa, sa_leaf.data(), sa_leaf.size() * 4);
    put(o_sb, sb_leaf.data(), sb_leaf.size() * 4);
    put(o_cq_ptr, cq_ptr.data(), cq_ptr.size() * 4);
    put(o_cq_leaf, cq_leaf.data(), cq_leaf.size() * 4);
    put(o_cq_coef, cq_coef.data(), cq_coef.size() * 8);
    put(o_lu_ptr, lu_ptr.data(), lu_ptr.size() * 4);
    put(o_lu_code, lu_code.data(), lu_code.size() * 4);
    put(o_lu_coef, lu_coef.data(), lu_coef.size() * 8);
    put(o_lv_ptr, lv_ptr.data(), lv_ptr.size() * 4);
    put(o_lv_code, lv_code.data(), lv_code.size() * 4);
    put(o_lv_coef, lv_coef.data(), lv_coef.size() * 8);
    put(o_lw_ptr, lw_ptr.data(), lw_ptr.size() * 4);
    put(o_lw_r, lw_r.data(), lw_r.size() * 4);
    put(o_lw_coef, lw_coef.data(), lw_coef.size() * 8);
    put(o_leaf_slot, leaf_slot.data(), leaf_slot.size() * 4);
    put(o_c_raw, c_coef_raw.data(), c_coef_raw.size() * 8);
    put(o_a_raw, p->a.coef.data(), p->a.coef.size() * 8);
    put(o_b_raw, p->b.coef.data(), p->b.coef.size() * 8);
    put(o_lu_i, lu_icoef.data(), lu_icoef.size() * 4);
    put(o_lv_i, lv_icoef.data(), lv_icoef.size() * 4);
    put(o_lw_i, lw_icoef.data(), lw_icoef.size() * 4);
    put(o_lvt, lvt_code.data(), lvt_code.size() * 4);

    void *blob = nullptr;
    cudaError_t e = cudaMalloc(&blob, bl.bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? FMM_ERR_NO_MEMORY : FMM_ERR_CUDA;
    }
    e = cudaMemcpy(blob, host.data(), bl.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(blob);
        return FMM_ERR_CUDA;
    }
    char *b = (char *)blob;
    DevicePlan &d = p->dev;
    d.blob = blob;
    d.a_ptr = (int *)(b + o_a_ptr); d.a_code = (int *)(b + o_a_code); d.a_coef = (double *)(b + o_a_coef);
    d.b_ptr = (int *)(b + o_b_ptr); d.b_code = (int *)(b + o_b_code); d.b_coef = (double *)(b + o_b_coef);
    d.c_ptr = (int *)(b + o_c_ptr); d.c_code = (int *)(b + o_c_code); d.c_coef = (double *)(b + o_c_coef);
    d.ua_code = (int *)(b + o_ua); d.ub_code = (int *)(b + o_ub);
    d.ua_ptr = d.ub_ptr = (int *)(b + o_uptr);
    d.u_one = (double *)(b + o_one);
    d.sa_leaf = (int *)(b + o_sa); d.sb_leaf = (int *)(b + o_sb);
    d.cq_ptr = (int *)(b + o_cq_ptr); d.cq_leaf = (int *)(b + o_cq_leaf); d.cq_coef = (double *)(b + o_cq_coef);
    d.lu_ptr = (int *)(b + o_lu_ptr); d.lu_code = (int *)(b + o_lu_code); d.lu_coef = (double *)(b + o_lu_coef);
    d.lv_ptr = (int *)(b + o_lv_ptr); d.lv_code = (int *)(b + o_lv_code); d.lv_coef = (double *)(b + o_lv_coef);
    d.lw_ptr = (int *)(b + o_lw_ptr); d.lw_r = (int *)(b + o_lw_r); d.lw_coef = (double *)(b + o_lw_coef);
    d.leaf_slot = (int *)(b + o_leaf_slot); d.c_coef_raw = (double *)(b + o_c_raw);
    d.a_coef_raw = (double *)(b + o_a_raw); d.b_coef_raw = (double *)(b + o_b_raw);
    d.lu_icoef = (int *)(b + o_lu_i); d.lv_icoef = (int *)(b + o_lv_i); d.lw_icoef = (int *)(b + o_lw_i);
    d.lvt_code = (int *)(b + o_lvt);
    return FMM_OK;
}

void free_plan_device(fmm_plan *p) {
    if (p->dev.blob) cudaFree(p->dev.blob);
    p->dev = DevicePlan{};
}

static bool parse_rational(const std::string &tok, double *out, bool *dyadic_ok) {
    const size_t slash = tok.find('/');
    char *end = nullptr;
    if (slash == std::string::npos) {
        long long v = std::strtoll(tok.c_str(), &end, 10);
        if (end == tok.c_str() || *end != '\0') return false;
        *out = (double)v;
        return true;
    }
    const std::string a = tok.substr(0, slash), b = tok.substr(slash + 1);
    long long num = std::strtoll(a.c_str(), &end, 10);
    if (end == a.c_str() || *end != '\0') return false;
    long long den = std::strtoll(b.c_str(), &end, 10);
    if (end == b.c_str() || *end != '\0' || den <= 0) return false;
    if ((den & (den - 1)) != 0) *dyadic_ok = false;
    *out = (double)num / (double)den;
    return true;
}

fmm_status parse_fmm_file(const char *path, int *M, int *K, int *N, int *R,
                          std::vector<double> *U, std::vector<double> *V,
                          std::vector<double> *W) {
    std::ifstream in(path);
    if (!in) return FMM_ERR_ARG;
    std::vector<std::string> lines;
    std::string ln;
    while (std::getline(in, ln)) {
        const size_t h = ln.find('#');
        if (h != std::string::npos) ln = ln.substr(0, h);
        size_t a = ln.find_first_not_of(" \t\r");
        if (a == std::string::npos) continue;
        size_t z = ln.find_last_not_of(" \t\r");
        lines.push_back(ln.substr(a, z - a + 1));
    }
    if (lines.empty()) return FMM_ERR_ARG;
    {
        std::istringstream hs(lines[0]);
        if (!(hs >> *M >> *K >> *N >> *R)) return FMM_ERR_ARG;
    }
    if (*M < 1 || *K < 1 || *N < 1 || *R < 1 || *M > 16 || *K > 16 || *N > 16 || *R > 4096)
        return FMM_ERR_ARG;
    size_t pos = 1;
    bool dy = true;
    const char *names[3] = {"U", "V", "W"};
    const int rows[3] = {*M * *K, *K * *N, *M * *N};
    std::vector<double> *outs[3] = {U, V, W};
    for (int blk = 0; blk < 3; ++blk) {
        if (pos >= lines.size() || lines[pos] != names[blk]) return FMM_ERR_ARG;
        ++pos;
        outs[blk]->assign((size_t)rows[blk] * *R, 0.0);
        for (int i = 0; i < rows[blk]; ++i, ++pos) {
            if (pos >= lines.size()) return FMM_ERR_ARG;
            std::istringstream rs(lines[pos]);
            std::string tok;
            int cnt = 0;
            while (rs >> tok) {
                if (cnt >= *R) return FMM_ERR_ARG;
                double v;
                if (!parse_rational(tok, &v, &dy)) return FMM_ERR_ARG;
                (*outs[blk])[(size_t)i * *R + cnt++] = v;
            }
            if (cnt != *R) return FMM_ERR_ARG;
        }
    }
    if (!dy) return FMM_ERR_UNSUPPORTED;
    return FMM_OK;
}

}  // namespace fmm
