// Domain tree (Section 2, Definition "Domain tree") and the padded slot map.
//
// Each node splits into 2^d children by halving its points along x, then
// each half along y (then z): sort by (coordinate, original index), lower
// half = first floor(n/2).  On a power-of-two grid of cell centres this is
// the paper's uniform 2^d partition of an ideal domain.  Child id
// c = b_0 + 2 b_1 + 4 b_2 (b_a = 1: upper half along axis a); children are
// stored in id order, so each node is a contiguous tree-order range.
//
// The GPU layout pads every leaf to m_pad slots (largest leaf rounded up to
// a multiple of 8, or 16 for e4m3 storage), which makes node n of level l the slot range
// [n * n_l, (n+1) * n_l) with n_l = m_pad 2^(d (L - l)).
#include <algorithm>
#include <cstdio>

#include "hm_internal.h"

namespace hm {

int tree_depth(int64_t N, int d, int leaf_size) {
    int L = 0;
    while (true) {
        const int64_t parts = (int64_t)1 << (d * L);
        if ((N + parts - 1) / parts <= leaf_size) return L;
        ++L;
    }
}

namespace {

struct Splitter {
    const double* pts;
    int d;
    std::vector<int64_t>& work;   // original indices, tree order being formed
    std::vector<int64_t> tmp;

    // Sort work[b, e) by (coordinate `axis`, original index).
    void sort_axis(int64_t b, int64_t e, int axis) {
        const double* P = pts;
        const int dd = d;
        std::sort(work.begin() + b, work.begin() + e, [P, dd, axis](int64_t u, int64_t v) {
            const double cu = P[u * dd + axis], cv = P[v * dd + axis];
            if (cu != cv) return cu < cv;
            return u < v;
        });
    }

    // Split node [b, e) into 2^d children; writes child begins/counts in id order.
    void split(int64_t b, int64_t e, int64_t* cbeg, int64_t* ccnt) {
        // parts in halving order: position bits b_0 ... b_{d-1}, b_0 most significant
        std::vector<int64_t> pb{b}, pe{e};
        for (int axis = 0; axis < d; ++axis) {
            std::vector<int64_t> nb, ne;
            for (size_t i = 0; i < pb.size(); ++i) {
                sort_axis(pb[i], pe[i], axis);
                const int64_t h = (pe[i] - pb[i]) / 2;
                nb.push_back(pb[i]);
                ne.push_back(pb[i] + h);
                nb.push_back(pb[i] + h);
                ne.push_back(pe[i]);
            }
            pb.swap(nb);
            pe.swap(ne);
        }
        // reorder the parts to child-id order c = sum_a b_a 2^a
        const int nc = 1 << d;
        tmp.assign(work.begin() + b, work.begin() + e);
        int64_t off = b;
        for (int c = 0; c < nc; ++c) {
            int pos = 0;
            for (int a = 0; a < d; ++a) pos |= ((c >> a) & 1) << (d - 1 - a);
            const int64_t n = pe[pos] - pb[pos];
            std::copy(tmp.begin() + (pb[pos] - b), tmp.begin() + (pe[pos] - b),
                      work.begin() + off);
            cbeg[c] = off;
            ccnt[c] = n;
            off += n;
        }
    }
};

}  // namespace

void build_tree(const double* points, int64_t N, int d, int leaf_size, int threads,
                int slot_multiple, Tree& t) {
    t.d = d;
    t.N = N;
    t.leaf_size = leaf_size;
    t.L = tree_depth(N, d, leaf_size);
    t.perm.resize(N);
    for (int64_t i = 0; i < N; ++i) t.perm[i] = i;
    t.beg.assign(t.L + 1, {});
    t.cnt.assign(t.L + 1, {});
    t.beg[0] = {0};
    t.cnt[0] = {N};
    const int nc = 1 << d;
    for (int l = 0; l < t.L; ++l) {
        const int64_t nodes = (int64_t)t.beg[l].size();
        t.beg[l + 1].assign(nodes * nc, 0);
        t.cnt[l + 1].assign(nodes * nc, 0);
        // nodes of one level touch disjoint ranges: split them in parallel
        parallel_for(nodes, threads, [&](int64_t j) {
            Splitter sp{points, d, t.perm, {}};
            sp.split(t.beg[l][j], t.beg[l][j] + t.cnt[l][j], &t.beg[l + 1][j * nc],
                     &t.cnt[l + 1][j * nc]);
        });
    }
    // padded slots
    int64_t mx = 0;
    for (int64_t c : t.cnt[t.L]) mx = std::max(mx, c);
    const int64_t q = slot_multiple > 8 ? slot_multiple : 8;
    t.m_pad = (int)std::max<int64_t>(q, (mx + q - 1) / q * q);
    const int64_t leaves = (int64_t)t.beg[t.L].size();
    t.Np = (int64_t)t.m_pad * leaves;
    t.slot.assign(N, -1);
    t.slot_src.assign(t.Np, -1);
    for (int64_t lf = 0; lf < leaves; ++lf) {
        for (int64_t a = 0; a < t.cnt[t.L][lf]; ++a) {
            const int64_t p = t.beg[t.L][lf] + a;
            const int64_t sl = lf * t.m_pad + a;
            t.slot[p] = sl;
            t.slot_src[sl] = t.perm[p];
        }
    }
}

}  // namespace hm

namespace hm {

void node_coords(int64_t i, int d, int l, int* c) {
    for (int a = 0; a < 3; ++a) c[a] = 0;
    for (int b = 0; b < l; ++b)
        for (int a = 0; a < d; ++a) c[a] |= (int)((i >> (d * b + a)) & 1) << b;
}

int64_t node_index(const int* c, int d, int l) {
    int64_t i = 0;
    for (int b = 0; b < l; ++b)
        for (int a = 0; a < d; ++a) i |= (int64_t)((c[a] >> b) & 1) << (d * b + a);
    return i;
}

void build_stencil(int d, Stencil& st) {
    st.d = d;
    st.nnb = d == 2 ? 9 : 27;
    st.nslot = (d == 2 ? 36 : 216) - st.nnb;
    const int classes = 1 << d;
    st.off.assign((size_t)classes * st.nslot * 3, 0);
    st.rev.assign((size_t)classes * st.nslot, -1);
    st.packed.assign((size_t)classes * st.nslot, 0);
    for (int p = 0; p < classes; ++p) {
        int q = 0;
        int dl[3] = {0, 0, 0};
        // increasing (delta_{d-1}, ..., delta_0): delta_0 fastest
        const int n = d == 2 ? 36 : 216;
        for (int e = 0; e < n; ++e) {
            int r = e;
            bool touch = true;
            for (int a = 0; a < d; ++a) {
                const int pa = (p >> a) & 1;
                dl[a] = -2 - pa + r % 6;
                r /= 6;
                if (dl[a] < -1 || dl[a] > 1) touch = false;
            }
            if (touch) continue;
            for (int a = 0; a < 3; ++a) st.off[((size_t)p * st.nslot + q) * 3 + a] = a < d ? dl[a] : 0;
            ++q;
        }
    }
    // reverse slots: node j = i + delta has class (p + delta) mod 2 per axis
    for (int p = 0; p < classes; ++p)
        for (int q = 0; q < st.nslot; ++q) {
            const int* o = &st.off[((size_t)p * st.nslot + q) * 3];
            int pj = 0;
            for (int a = 0; a < d; ++a) pj |= (((p >> a) & 1) + o[a]) & 1 ? 1 << a : 0;
            for (int q2 = 0; q2 < st.nslot; ++q2) {
                const int* o2 = &st.off[((size_t)pj * st.nslot + q2) * 3];
                bool same = true;
                for (int a = 0; a < d; ++a) same = same && o2[a] == -o[a];
                if (same) {
                    st.rev[(size_t)p * st.nslot + q] = q2;
                    break;
                }
            }
            int pk = st.rev[(size_t)p * st.nslot + q] << 12;
            for (int a = 0; a < 3; ++a) pk |= (o[a] + 4) << (4 * a);
            st.packed[(size_t)p * st.nslot + q] = pk;
        }
}

int stencil_slot(const Stencil& st, const int* ci, const int* delta) {
    int p = 0;
    for (int a = 0; a < st.d; ++a) p |= (ci[a] & 1) << a;
    for (int q = 0; q < st.nslot; ++q) {
        const int* o = &st.off[((size_t)p * st.nslot + q) * 3];
        bool same = true;
        for (int a = 0; a < st.d; ++a) same = same && o[a] == delta[a];
        if (same) return q;
    }
    return -1;
}

}  // namespace hm
