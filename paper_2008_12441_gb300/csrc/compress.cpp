// Block structure (Definition def:hmat, weak admissibility), block contents
// and the flattened device layout of every level.
//
// The paper leaves construction out of scope (end of Section 2) and fills
// its benchmark matrices with random numbers (Section 5.1).  This builder
// offers: truncated SVD (orthogonal subspace iteration run to convergence,
// Golub & Van Loan Sec. 8.2.4), randomized SVD (Halko, Martinsson, Tropp
// 2011: range finder with q power iterations) and counter-based random
// fill.  Factors are U = Q U_B S_r and V = V_B,r (V orthonormal).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <new>

#include "hm_internal.h"
#include "philox_hm.h"

namespace hm {

// ----------------------------------------------------------- small dense LA
namespace {

struct Mat {  // column-major m x n
    int64_t m = 0, n = 0;
    std::vector<double> a;
    Mat() = default;
    Mat(int64_t m_, int64_t n_) : m(m_), n(n_), a((size_t)(m_ * n_), 0.0) {}
    double* col(int64_t j) { return a.data() + j * m; }
    const double* col(int64_t j) const { return a.data() + j * m; }
    double& operator()(int64_t i, int64_t j) { return a[j * m + i]; }
    double operator()(int64_t i, int64_t j) const { return a[j * m + i]; }
};

// Thin Q (m x n, n <= m) of the Householder QR of A.
Mat householder_q(Mat A) {
    const int64_t m = A.m, n = A.n;
    std::vector<std::vector<double>> vs(n);
    for (int64_t k = 0; k < n; ++k) {
        double* x = A.col(k) + k;
        const int64_t len = m - k;
        double nrm = 0.0;
        for (int64_t i = 0; i < len; ++i) nrm += x[i] * x[i];
        nrm = std::sqrt(nrm);
        std::vector<double> v(x, x + len);
        if (nrm == 0.0) {
            vs[k].clear();
            continue;
        }
        v[0] += (x[0] >= 0 ? nrm : -nrm);
        double vn = 0.0;
        for (double e : v) vn += e * e;
        vn = std::sqrt(vn);
        for (double& e : v) e /= vn;
        for (int64_t j = k; j < n; ++j) {
            double* c = A.col(j) + k;
            double dot = 0.0;
            for (int64_t i = 0; i < len; ++i) dot += v[i] * c[i];
            for (int64_t i = 0; i < len; ++i) c[i] -= 2.0 * dot * v[i];
        }
        vs[k] = std::move(v);
    }
    Mat Q(m, n);
    for (int64_t j = 0; j < n; ++j) Q(j, j) = 1.0;
    for (int64_t k = n - 1; k >= 0; --k) {
        if (vs[k].empty()) continue;
        const std::vector<double>& v = vs[k];
        const int64_t len = m - k;
        for (int64_t j = 0; j < n; ++j) {
            double* c = Q.col(j) + k;
            double dot = 0.0;
            for (int64_t i = 0; i < len; ++i) dot += v[i] * c[i];
            if (dot == 0.0) continue;
            for (int64_t i = 0; i < len; ++i) c[i] -= 2.0 * dot * v[i];
        }
    }
    return Q;
}

// C = A^T B  (A: m x p, B: m x q) -> p x q
Mat atb(const Mat& A, const Mat& B) {
    Mat C(A.n, B.n);
    for (int64_t j = 0; j < B.n; ++j)
        for (int64_t i = 0; i < A.n; ++i) {
            const double* a = A.col(i);
            const double* b = B.col(j);
            double s = 0.0;
            for (int64_t k = 0; k < A.m; ++k) s += a[k] * b[k];
            C(i, j) = s;
        }
    return C;
}

// C = A B  (A: m x p, B: p x q) -> m x q
Mat ab(const Mat& A, const Mat& B) {
    Mat C(A.m, B.n);
    for (int64_t j = 0; j < B.n; ++j) {
        double* c = C.col(j);
        for (int64_t k = 0; k < A.n; ++k) {
            const double bkj = B(k, j);
            if (bkj == 0.0) continue;
            const double* a = A.col(k);
            for (int64_t i = 0; i < A.m; ++i) c[i] += a[i] * bkj;
        }
    }
    return C;
}

// One-sided (Hestenes) Jacobi SVD of a square or tall W (m x n):
// W = Ul diag(S) Vr^T, singular values sorted descending.  Columns of Ul
// with S = 0 are zero.
void jacobi_svd(Mat W, Mat& Ul, std::vector<double>& S, Mat& Vr) {
    const int64_t m = W.m, n = W.n;
    Mat J(n, n);
    for (int64_t i = 0; i < n; ++i) J(i, i) = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        bool rotated = false;
        for (int64_t p = 0; p < n - 1; ++p)
            for (int64_t q = p + 1; q < n; ++q) {
                double al = 0, be = 0, ga = 0;
                const double* wp = W.col(p);
                const double* wq = W.col(q);
                for (int64_t i = 0; i < m; ++i) {
                    al += wp[i] * wp[i];
                    be += wq[i] * wq[i];
                    ga += wp[i] * wq[i];
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
                rotated = true;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) /
                                 (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                double* xp = W.col(p);
                double* xq = W.col(q);
                for (int64_t i = 0; i < m; ++i) {
                    const double u = xp[i], v = xq[i];
                    xp[i] = c * u - s * v;
                    xq[i] = s * u + c * v;
                }
                double* jp = J.col(p);
                double* jq = J.col(q);
                for (int64_t i = 0; i < n; ++i) {
                    const double u = jp[i], v = jq[i];
                    jp[i] = c * u - s * v;
                    jq[i] = s * u + c * v;
                }
            }
        if (!rotated) break;
    }
    std::vector<double> nr(n);
    for (int64_t j = 0; j < n; ++j) {
        double s = 0;
        for (int64_t i = 0; i < m; ++i) s += W(i, j) * W(i, j);
        nr[j] = std::sqrt(s);
    }
    std::vector<int64_t> ord(n);
    for (int64_t j = 0; j < n; ++j) ord[j] = j;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return nr[a] > nr[b]; });
    Ul = Mat(m, n);
    Vr = Mat(n, n);
    S.assign(n, 0.0);
    for (int64_t k = 0; k < n; ++k) {
        const int64_t j = ord[k];
        S[k] = nr[j];
        if (nr[j] > 0)
            for (int64_t i = 0; i < m; ++i) Ul(i, k) = W(i, j) / nr[j];
        for (int64_t i = 0; i < n; ++i) Vr(i, k) = J(i, j);
    }
}

// ------------------------------------------------------------ kernel block
struct KBlock {
    int kernel, d;
    const double* pt;      // target points (tree order), nt x d
    const int64_t* it;     // their original indices
    int64_t nt;
    const double* ps;
    const int64_t* is;
    int64_t ns;
    std::atomic<int>* bad;

    double eval(int64_t a, int64_t b) const {
        if (it[a] == is[b]) return 1.0;
        double r2 = 0.0;
        for (int k = 0; k < d; ++k) {
            const double df = pt[a * d + k] - ps[b * d + k];
            r2 += df * df;
        }
        const double r = std::sqrt(r2);
        if (r == 0.0) {
            bad->store(1);
            return 0.0;
        }
        if (kernel == HMAT_K_LOG2D) return -std::log(r);
        return 1.0 / (4.0 * M_PI * r);
    }
    Mat dense() const {
        Mat A(nt, ns);
        for (int64_t b = 0; b < ns; ++b)
            for (int64_t a = 0; a < nt; ++a) A(a, b) = eval(a, b);
        return A;
    }
};

// Kernel block as an operator: materialised when small, evaluated row tile
// by row tile otherwise.
struct KOp {
    const KBlock& kb;
    Mat A;
    bool mat;
    explicit KOp(const KBlock& k) : kb(k), mat(k.nt * k.ns <= (int64_t)8 << 20) {
        if (mat) A = kb.dense();
    }
    Mat apply(const Mat& M) const {  // A M: nt x q
        if (mat) return ab(A, M);
        Mat Y(kb.nt, M.n);
        const int64_t TR = 64;
        std::vector<double> tile((size_t)(TR * kb.ns));
        for (int64_t a0 = 0; a0 < kb.nt; a0 += TR) {
            const int64_t na = std::min(TR, kb.nt - a0);
            for (int64_t b = 0; b < kb.ns; ++b)
                for (int64_t a = 0; a < na; ++a) tile[b * na + a] = kb.eval(a0 + a, b);
            for (int64_t j = 0; j < M.n; ++j) {
                const double* mj = M.col(j);
                double* y = Y.col(j) + a0;
                for (int64_t b = 0; b < kb.ns; ++b) {
                    const double w = mj[b];
                    const double* t = &tile[b * na];
                    for (int64_t a = 0; a < na; ++a) y[a] += t[a] * w;
                }
            }
        }
        return Y;
    }
    Mat apply_t(const Mat& M) const {  // A^T M: ns x q
        if (mat) return atb(A, M);
        Mat Z(kb.ns, M.n);
        const int64_t TR = 64;
        std::vector<double> tile((size_t)(TR * kb.ns));
        for (int64_t a0 = 0; a0 < kb.nt; a0 += TR) {
            const int64_t na = std::min(TR, kb.nt - a0);
            for (int64_t b = 0; b < kb.ns; ++b)
                for (int64_t a = 0; a < na; ++a) tile[b * na + a] = kb.eval(a0 + a, b);
            for (int64_t j = 0; j < M.n; ++j) {
                const double* mj = M.col(j) + a0;
                double* z = Z.col(j);
                for (int64_t b = 0; b < kb.ns; ++b) {
                    const double* t = &tile[b * na];
                    double s = 0.0;
                    for (int64_t a = 0; a < na; ++a) s += t[a] * mj[a];
                    z[b] += s;
                }
            }
        }
        return Z;
    }
};

Mat sketch(uint64_t seed, int level, int64_t t, int64_t s, int64_t ns, int64_t ell) {
    Mat Om(ns, ell);
    for (int64_t c = 0; c < ell; ++c)
        for (int64_t b = 0; b < ns; ++b)
            Om(b, c) = rand_entry(seed, RAND_SKETCH, level, (uint32_t)t, (uint32_t)s,
                                  (uint32_t)b, (uint32_t)c);
    return Om;
}

int rank_of(const std::vector<double>& S, int rank, double tol, int64_t cap) {
    if (rank > 0) return (int)std::min<int64_t>(rank, cap);
    if (S.empty() || S[0] == 0.0) return 0;
    int64_t k = 0;
    while (k < (int64_t)S.size() && k < cap && S[k] > tol * S[0]) ++k;
    return (int)k;
}

// Factors from a range basis Q (nt x ell): B^T = A^T Q = Q2 R, R = W S J^T,
// so B = J S (Q2 W)^T: U = Q J_r S_r, V = (Q2 W)_r.
void factors_from_bt(const Mat& Q, const Mat& Bt, int64_t nt, int64_t ns, int rank, double tol,
                     Mat& U, Mat& V, int& rb) {
    Mat Q2 = householder_q(Bt);
    Mat R = atb(Q2, Bt);     // ell x ell
    Mat W, J;
    std::vector<double> S;
    jacobi_svd(R, W, S, J);
    rb = rank_of(S, rank, tol, std::min<int64_t>(Q.n, std::min(nt, ns)));
    U = Mat(nt, rb);
    V = Mat(ns, rb);
    Mat QJ = ab(Q, J);       // nt x ell
    Mat Q2W = ab(Q2, W);     // ns x ell
    for (int64_t c = 0; c < rb; ++c) {
        for (int64_t a = 0; a < nt; ++a) U(a, c) = QJ(a, c) * S[c];
        for (int64_t b = 0; b < ns; ++b) V(b, c) = Q2W(b, c);
    }
}

void factors_from_range(const KOp& op, const Mat& Q, int rank, double tol, Mat& U, Mat& V,
                        int& rb) {
    factors_from_bt(Q, op.apply_t(Q), op.kb.nt, op.kb.ns, rank, tol, U, V, rb);
}

void rsvd_block(const KOp& op, uint64_t seed, int level, int64_t t, int64_t s, int rank,
                double tol, int p, int q, Mat& U, Mat& V, int& rb) {
    const int64_t cap = std::min(op.kb.nt, op.kb.ns);
    const int64_t ell = std::min<int64_t>((rank > 0 ? rank : cap) + p, cap);
    Mat Q = householder_q(op.apply(sketch(seed, level, t, s, op.kb.ns, ell)));
    for (int it = 0; it < q; ++it) Q = householder_q(op.apply(householder_q(op.apply_t(Q))));
    factors_from_range(op, Q, rank, tol, U, V, rb);
}

// Truncated SVD by orthogonal subspace iteration, iterated until the rank-r
// product stops changing (checked on two probe vectors) to 1e-15.
void tsvd_block(const KOp& op, uint64_t seed, int level, int64_t t, int64_t s, int rank,
                double tol, Mat& U, Mat& V, int& rb) {
    const int64_t cap = std::min(op.kb.nt, op.kb.ns);
    const int64_t want = rank > 0 ? rank : cap;
    const int64_t ell = std::min<int64_t>(cap, want + std::max<int64_t>(want, 8));
    Mat Q = householder_q(op.apply(sketch(seed, level, t, s, op.kb.ns, ell)));
    Mat probe = sketch(seed ^ 0x5bd1e995ull, level, t, s, op.kb.ns, 2);
    Mat prev;
    for (int it = 0; it < 64; ++it) {
        factors_from_range(op, Q, rank, tol, U, V, rb);
        Mat cur = ab(U, atb(V, probe));  // (U V^T) probe
        if (ell == cap && it == 0) break; // full range: exact in one pass
        if (it > 0 && prev.n == cur.n && prev.m == cur.m) {
            double dn = 0, nn = 0;
            for (size_t i = 0; i < cur.a.size(); ++i) {
                dn += (cur.a[i] - prev.a[i]) * (cur.a[i] - prev.a[i]);
                nn += cur.a[i] * cur.a[i];
            }
            if (dn <= 1e-30 * nn) break;
        }
        prev = cur;
        Q = householder_q(op.apply(householder_q(op.apply_t(Q))));
    }
}

struct LRBlock {
    int64_t i, j;   // target / source node of the level
    int qu, qv;     // slot of source j at target i (U), of target i at source j (V)
    int rb = 0;
    Mat U, V;       // nt x rb, ns x rb
};

// Randomized SVD of every block of one level with the kernel-block products
// on the GPU (same steps as rsvd_block; QR and SVD stay on the host).
int rsvd_level_gpu(GpuSketch* gs, std::vector<LRBlock>& bl, int l, const Tree& tr,
                   const BuildParams& bp) {
    const size_t n = bl.size();
    std::vector<int64_t> ell(n);
    int ellmax = 0;
    for (size_t b = 0; b < n; ++b) {
        const int64_t nt = tr.cnt[l][bl[b].i], ns = tr.cnt[l][bl[b].j];
        const int64_t cap = std::min(nt, ns);
        ell[b] = std::min<int64_t>((bp.rank > 0 ? bp.rank : cap) + bp.oversample, cap);
        ellmax = std::max<int>(ellmax, (int)ell[b]);
    }
    if (ellmax == 0) return HMAT_OK;
    // one batched product: Out_b = A_b M_b (transpose: A_b^T M_b)
    auto run = [&](bool transpose, const std::vector<Mat>& Ms, std::vector<Mat>& Out) -> int {
        std::vector<SketchTask> tasks(n);
        int64_t moff = 0, yoff = 0;
        for (size_t b = 0; b < n; ++b) {
            const int64_t bi = tr.beg[l][bl[b].i], ni = tr.cnt[l][bl[b].i];
            const int64_t bj = tr.beg[l][bl[b].j], nj = tr.cnt[l][bl[b].j];
            SketchTask& t = tasks[b];
            t.row0 = transpose ? bj : bi;
            t.nrows = transpose ? nj : ni;
            t.col0 = transpose ? bi : bj;
            t.ncols = transpose ? ni : nj;
            t.m_off = moff;
            t.y_off = yoff;
            moff += t.ncols * ellmax;
            yoff += t.nrows * ellmax;
        }
        std::vector<float> M((size_t)moff, 0.f);
        std::vector<double> Y((size_t)yoff, 0.0);
        parallel_for((int64_t)n, bp.threads, [&](int64_t b) {
            const Mat& m = Ms[(size_t)b];
            for (int64_t r = 0; r < m.m; ++r)
                for (int64_t c = 0; c < m.n; ++c)
                    M[(size_t)(tasks[(size_t)b].m_off + r * ellmax + c)] = (float)m(r, c);
        });
        int rc = gpu_sketch_apply(gs, tasks, ellmax, M, Y);
        if (rc) return rc;
        Out.resize(n);
        parallel_for((int64_t)n, bp.threads, [&](int64_t b) {
            const SketchTask& t = tasks[(size_t)b];
            Mat o(t.nrows, ell[(size_t)b]);
            for (int64_t r = 0; r < t.nrows; ++r)
                for (int64_t c = 0; c < o.n; ++c) o(r, c) = Y[(size_t)(t.y_off + r * ellmax + c)];
            Out[(size_t)b] = std::move(o);
        });
        return HMAT_OK;
    };
    std::vector<Mat> Q(n), W(n);
    parallel_for((int64_t)n, bp.threads, [&](int64_t b) {
        W[(size_t)b] = sketch(bp.seed, l, bl[(size_t)b].i, bl[(size_t)b].j,
                              tr.cnt[l][bl[(size_t)b].j], ell[(size_t)b]);
    });
    int rc;
    auto orth_all = [&](std::vector<Mat>& in, std::vector<Mat>& out) {
        parallel_for((int64_t)n, bp.threads, [&](int64_t b) {
            out[(size_t)b] = householder_q(std::move(in[(size_t)b]));
        });
    };
    std::vector<Mat> Y;
    if ((rc = run(false, W, Y))) return rc;
    orth_all(Y, Q);
    for (int it = 0; it < bp.power_iters; ++it) {
        if ((rc = run(true, Q, Y))) return rc;
        orth_all(Y, W);
        if ((rc = run(false, W, Y))) return rc;
        orth_all(Y, Q);
    }
    std::vector<Mat> Bt;
    if ((rc = run(true, Q, Bt))) return rc;
    parallel_for((int64_t)n, bp.threads, [&](int64_t b) {
        LRBlock& blk = bl[(size_t)b];
        factors_from_bt(Q[(size_t)b], Bt[(size_t)b], tr.cnt[l][blk.i], tr.cnt[l][blk.j], bp.rank,
                        bp.tol, blk.U, blk.V, blk.rb);
    });
    return HMAT_OK;
}

}  // namespace

double block_uniform(uint64_t seed, int kind, int level, uint32_t t, uint32_t s,
                     uint32_t row, uint32_t col) {
    return rand_entry(seed, kind, level, t, s, row, col);
}

void layout_workspace(Geometry& g) {
    // partial-sum workspace: node sums, then per-tile partials and arrival
    // counters for the levels whose nodes span several project tiles
    int64_t t_off = 0, c_off = 0;
    for (int l = 1; l <= g.nf; ++l) {
        LevelGeom& lg = g.lv[l];
        const int64_t sr = (int64_t)g.s * lg.r;
        lg.fin_off = t_off;
        t_off += lg.nodes * sr;
        if (lg.nsub > 1) {
            lg.part_off = t_off;
            t_off += (g.Np / g.tile_p) * sr;
            lg.cnt_off = c_off;
            c_off += lg.nodes;
        }
    }
    g.counters = c_off;
    g.t_per_rhs = t_off;
}

bool random_fill_on_device_ok(const Tree& tr, const BuildParams& bp) {
    if (bp.method != HMAT_RANDOM_FILL || bp.adm != 0 || tr.L < 1 || tr.Np != tr.N) return false;
    for (int64_t c : tr.cnt[tr.L])
        if (c != tr.m_pad) return false;
    return true;
}

// Project tile: m_pad * 2^a slots, about 256, at most the whole tree; at
// most one near-field group of G slots when G is a multiple of 128 (the
// tensor-core kernels take whole tiles per group).
static int64_t project_tile(int64_t m_pad, int64_t Np, int64_t G) {
    int64_t tp = m_pad;
    while (tp * 2 <= 256 && tp * 2 <= Np && (G % 128 != 0 || tp * 2 <= G)) tp *= 2;
    return tp;
}

int random_fill_layout(const Tree& tr, const BuildParams& bp, Geometry& g, Master& m) {
    const int d = tr.d, nc = 1 << d;
    g.d = d;
    g.adm = 0;
    g.s = nc - 1;
    g.nnb = 1;
    g.L = tr.L;
    g.m_pad = tr.m_pad;
    g.Np = tr.Np;
    g.nf = bp.leaf_lowrank ? tr.L : tr.L - 1;
    g.tile_p = project_tile(g.m_pad, g.Np, g.Np >> (d * g.nf));
    g.lv.assign(g.nf + 1, LevelGeom{});
    int64_t fac_off = 0;
    m.factor_entries = 0;
    m.lowrank_blocks = 0;
    for (int l = 1; l <= g.nf; ++l) {
        LevelGeom& lg = g.lv[l];
        lg.level = l;
        lg.nodes = (int64_t)1 << (d * l);
        lg.n = g.Np >> (d * l);
        lg.r = (int)std::min<int64_t>(bp.rank, lg.n);     // full leaves: every block n_l x n_l
        lg.nsub = lg.n > g.tile_p ? (int)(lg.n / g.tile_p) : 1;
        lg.fac_off = fac_off;
        fac_off += (int64_t)g.s * lg.r * g.Np;
        const int64_t blocks = lg.nodes * (nc - 1);
        m.lowrank_blocks += blocks;
        m.factor_entries += blocks * 2 * lg.n * lg.r;
    }
    layout_workspace(g);
    g.fac_entries = fac_off;
    g.groups = (int64_t)1 << (d * g.nf);
    g.G = g.Np >> (d * g.nf);
    g.dense_entries = g.groups * g.G * g.G;
    m.dense_entries = g.dense_entries;
    m.dense_blocks = bp.leaf_lowrank ? g.groups : g.groups * nc * nc;
    return HMAT_OK;
}

int compress_all(const Tree& tr, const double* pts, const BuildParams& bp, Geometry& g,
                 Master& m) {
    const int d = tr.d;
    const int nc = 1 << d;
    const bool std_adm = bp.adm == 1;
    Stencil st;
    if (std_adm) build_stencil(d, st);
    g.d = d;
    g.adm = bp.adm;
    g.s = std_adm ? st.nslot : nc - 1;
    g.nnb = std_adm ? st.nnb : 1;
    g.L = tr.L;
    g.m_pad = tr.m_pad;
    g.Np = tr.Np;
    g.nf = (tr.L == 0) ? 0 : (bp.leaf_lowrank ? tr.L : tr.L - 1);
    g.tile_p = project_tile(g.m_pad, g.Np, g.Np >> (d * g.nf));
    std::atomic<int> bad{0};
    std::vector<int64_t> iperm(tr.perm);  // original index of tree position
    g.lv.assign(g.nf + 1, LevelGeom{});
    std::vector<std::vector<LRBlock>> blocks(g.nf + 1);
    int64_t fac_off = 0;
    m.factor_entries = 0;
    m.lowrank_blocks = 0;
    for (int l = 1; l <= g.nf; ++l) {
        LevelGeom& lg = g.lv[l];
        lg.level = l;
        lg.nodes = (int64_t)1 << (d * l);
        lg.n = g.Np >> (d * l);
        const int64_t parents = lg.nodes / nc;
        std::vector<LRBlock>& bl = blocks[l];
        if (!std_adm) {
            // weak: every ordered pair of distinct siblings
            bl.resize((size_t)(parents * nc * (nc - 1)));
            for (int64_t P = 0; P < parents; ++P) {
                int64_t k = P * nc * (nc - 1);
                for (int ci = 0; ci < nc; ++ci)
                    for (int cj = 0; cj < nc; ++cj) {
                        if (ci == cj) continue;
                        LRBlock& b = bl[(size_t)k++];
                        b.i = P * nc + ci;
                        b.j = P * nc + cj;
                        b.qv = ci < cj ? ci : ci - 1;
                        b.qu = cj < ci ? cj : cj - 1;
                    }
            }
        } else if (l >= 2) {
            // standard: the interaction list of every node (level 1 has none:
            // the root's children all touch)
            const int side = 1 << l;
            for (int64_t i = 0; i < lg.nodes; ++i) {
                int ci[3];
                node_coords(i, d, l, ci);
                int p = 0;
                for (int a = 0; a < d; ++a) p |= (ci[a] & 1) << a;
                for (int q = 0; q < st.nslot; ++q) {
                    const int* o = &st.off[((size_t)p * st.nslot + q) * 3];
                    int cj[3] = {0, 0, 0};
                    bool in = true;
                    for (int a = 0; a < d; ++a) {
                        cj[a] = ci[a] + o[a];
                        in = in && cj[a] >= 0 && cj[a] < side;
                    }
                    if (!in) continue;
                    LRBlock b;
                    b.i = i;
                    b.j = node_index(cj, d, l);
                    b.qu = q;
                    b.qv = st.rev[(size_t)p * st.nslot + q];
                    bl.push_back(std::move(b));
                }
            }
        }
        const bool on_gpu = bp.gpu && bp.method == HMAT_RSVD;
        if (on_gpu) {
            int rc = rsvd_level_gpu(bp.gpu, bl, l, tr, bp);
            if (rc) return rc;
        }
        if (!on_gpu) parallel_for((int64_t)bl.size(), bp.threads, [&](int64_t bi) {
            LRBlock& b = bl[(size_t)bi];
            const int64_t nt = tr.cnt[l][b.i], ns = tr.cnt[l][b.j];
            const int64_t bt = tr.beg[l][b.i], bs = tr.beg[l][b.j];
            if (bp.method == HMAT_RANDOM_FILL) {
                b.rb = (int)std::min<int64_t>(bp.rank, std::min(nt, ns));
                b.U = Mat(nt, b.rb);
                b.V = Mat(ns, b.rb);
                const double su = rand_scale(b.rb), sv = rand_scale(ns);
                for (int c = 0; c < b.rb; ++c) {
                    for (int64_t a = 0; a < nt; ++a)
                        b.U(a, c) = su * rand_entry(bp.seed, RAND_U, l, (uint32_t)b.i,
                                                    (uint32_t)b.j, (uint32_t)a, (uint32_t)c);
                    for (int64_t a = 0; a < ns; ++a)
                        b.V(a, c) = sv * rand_entry(bp.seed, RAND_V, l, (uint32_t)b.i,
                                                    (uint32_t)b.j, (uint32_t)a, (uint32_t)c);
                }
                return;
            }
            if (nt == 0 || ns == 0) {
                b.rb = 0;
                b.U = Mat(nt, 0);
                b.V = Mat(ns, 0);
                return;
            }
            KBlock kb{bp.kernel, d, pts + bt * d, iperm.data() + bt, nt,
                      pts + bs * d, iperm.data() + bs, ns, &bad};
            KOp op(kb);
            if (bp.method == HMAT_TSVD)
                tsvd_block(op, bp.seed, l, b.i, b.j, bp.rank, bp.tol, b.U, b.V, b.rb);
            else
                rsvd_block(op, bp.seed, l, b.i, b.j, bp.rank, bp.tol, bp.oversample,
                           bp.power_iters, b.U, b.V, b.rb);
        });
        if (bad.load()) {
            set_error("hmat_build: two distinct points coincide");
            return HMAT_EINVAL;
        }
        int r = 0;
        for (const LRBlock& b : bl) {
            r = std::max(r, b.rb);
            m.factor_entries += (int64_t)(b.U.m + b.V.m) * b.rb;
        }
        m.lowrank_blocks += (int64_t)bl.size();
        lg.r = r;
        lg.nsub = lg.n > g.tile_p ? (int)(lg.n / g.tile_p) : 1;
        lg.fac_off = fac_off;
        fac_off += (int64_t)g.s * r * g.Np;
    }
    layout_workspace(g);
    g.fac_entries = fac_off;
    // scatter low-rank factors into the level layout
    if (injected_alloc_failure()) throw std::bad_alloc();
    m.U.assign((size_t)g.fac_entries, 0.0);
    m.V.assign((size_t)g.fac_entries, 0.0);
    for (int l = 1; l <= g.nf; ++l) {
        const LevelGeom& lg = g.lv[l];
        const int64_t sr = (int64_t)g.s * lg.r;
        parallel_for((int64_t)blocks[l].size(), bp.threads, [&](int64_t bi) {
            const LRBlock& b = blocks[l][(size_t)bi];
            const int qv = b.qv, qu = b.qu;
            const int64_t bt = tr.beg[l][b.i], bs = tr.beg[l][b.j];
            double* Vj = m.V.data() + lg.fac_off + b.j * sr * lg.n;
            double* Ui = m.U.data() + lg.fac_off + b.i * sr * lg.n;
            for (int c = 0; c < b.rb; ++c) {
                double* vc = Vj + (int64_t)(qv * lg.r + c) * lg.n;
                for (int64_t a = 0; a < b.V.m; ++a)
                    vc[tr.slot[bs + a] - b.j * lg.n] = b.V(a, c);
                double* uc = Ui + (int64_t)(qu * lg.r + c) * lg.n;
                for (int64_t a = 0; a < b.U.m; ++a)
                    uc[tr.slot[bt + a] - b.i * lg.n] = b.U(a, c);
            }
        });
        blocks[l].clear();
        blocks[l].shrink_to_fit();
    }
    // dense near-field groups: nodes of level nf.  Group g's block holds,
    // for each of its nnb source groups k (weak: g itself; standard: the
    // 3^d boxes touching g, offsets in increasing (e_{d-1}, ..., e_0) order,
    // zero columns where a box lies outside the domain), G columns stored
    // transposed: column k G + b contiguous over the target slots.
    g.groups = (int64_t)1 << (d * g.nf);
    g.G = g.Np >> (d * g.nf);
    g.dense_entries = g.groups * g.nnb * g.G * g.G;
    if (injected_alloc_failure()) throw std::bad_alloc();
    m.D.assign((size_t)g.dense_entries, 0.0);
    const bool leaf_pairs = (tr.L >= 1 && !bp.leaf_lowrank);  // reading A: leaves under touching parents
    // source group of group gi in near-field slot k (-1: outside the domain)
    auto src_group = [&](int64_t gi, int k) -> int64_t {
        if (!std_adm) return gi;
        int c[3];
        node_coords(gi, d, g.nf, c);
        const int side = 1 << g.nf;
        int r = k;
        for (int a = 0; a < d; ++a) {
            c[a] += r % 3 - 1;
            r /= 3;
            if (c[a] < 0 || c[a] >= side) return -1;
        }
        return node_index(c, d, g.nf);
    };
    m.dense_blocks = 0;
    m.dense_entries = 0;
    for (int64_t gi = 0; gi < g.groups; ++gi)
        for (int k = 0; k < g.nnb; ++k) {
            const int64_t gs = src_group(gi, k);
            if (gs < 0) continue;
            m.dense_entries += tr.cnt[g.nf][gi] * tr.cnt[g.nf][gs];
            m.dense_blocks += leaf_pairs ? nc * nc : 1;
        }
    // leaf and local index of a group's k-th point (tree order)
    auto leaves_of = [&](int64_t gi, std::vector<int64_t>& leaf, std::vector<int64_t>& loc) {
        const int64_t n = tr.cnt[g.nf][gi];
        leaf.assign(n, 0);
        loc.assign(n, 0);
        if (leaf_pairs) {
            int64_t k = 0;
            for (int c = 0; c < nc; ++c) {
                const int64_t lf = gi * nc + c;
                for (int64_t a = 0; a < tr.cnt[tr.L][lf]; ++a, ++k) {
                    leaf[k] = lf;
                    loc[k] = a;
                }
            }
        } else {
            for (int64_t k = 0; k < n; ++k) {
                leaf[k] = gi;
                loc[k] = k;
            }
        }
    };
    parallel_for(g.groups, bp.threads, [&](int64_t gi) {
        const int64_t b0 = tr.beg[g.nf][gi], n = tr.cnt[g.nf][gi];
        const int64_t s0 = gi * g.G;
        std::vector<int64_t> leaf, loc, sleaf, sloc;
        leaves_of(gi, leaf, loc);
        const int lev = leaf_pairs ? tr.L : g.nf;
        for (int k = 0; k < g.nnb; ++k) {
            const int64_t gs = src_group(gi, k);
            if (gs < 0) continue;
            const int64_t c0 = tr.beg[g.nf][gs], ns = tr.cnt[g.nf][gs], t0 = gs * g.G;
            leaves_of(gs, sleaf, sloc);
            double* Dg = m.D.data() + (gi * g.nnb + k) * g.G * g.G;
            KBlock kb{bp.kernel, d, pts + b0 * d, iperm.data() + b0, n,
                      pts + c0 * d, iperm.data() + c0, ns, &bad};
            for (int64_t bcol = 0; bcol < ns; ++bcol) {
                const int64_t sb = tr.slot[c0 + bcol] - t0;
                const double sc = rand_scale(leaf_pairs ? tr.cnt[tr.L][sleaf[bcol]] : ns);
                for (int64_t a = 0; a < n; ++a) {
                    const int64_t sa = tr.slot[b0 + a] - s0;
                    double v;
                    if (bp.method == HMAT_RANDOM_FILL)
                        v = sc * rand_entry(bp.seed, RAND_D, lev, (uint32_t)leaf[a],
                                            (uint32_t)sleaf[bcol], (uint32_t)loc[a],
                                            (uint32_t)sloc[bcol]);
                    else
                        v = kb.eval(a, bcol);
                    Dg[sb * g.G + sa] = v;
                }
            }
        }
    });
    if (bad.load()) {
        set_error("hmat_build: two distinct points coincide");
        return HMAT_EINVAL;
    }
    return HMAT_OK;
}

}  // namespace hm
