// Plan: monomial tables, the closed-form rank, the index table of the Gram
// identity (Eq. 1), workspace layout and device residency.
//
// Canonical order (Sec. 1.1, printed example for n = d = 2): higher total
// degree first, then lexicographically larger exponent tuple first.  The
// tables are generated directly in that order (degree D from high to low,
// each exponent from high to low), and positions are computed in closed form:
// with suffix sums S_j(g) = g_j + ... + g_n (1-based j),
//
//   rank(g) = sum_{s = S_1 + 1}^{2d} C(s + n - 1, n - 1)          (higher degrees)
//           + sum_{j = 2}^{n} [S_j > 0] C(S_j + n - j, n - j + 1)  (larger tuples of
//                                                                   the same degree)
//
// The second sum counts, position by position, the tuples that agree with g
// before position j-1 and are larger there (a hockey-stick sum of binomials).
// Because S_j(a + b) = S_j(a) + S_j(b), the index of a product of two
// monomials is separable:  idx(a, b) = sum_j phi_j[S_j(a) + S_j(b)].
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

namespace sos {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    cudaGetLastError();  // clear a sticky launch error where possible
    return e == cudaErrorMemoryAllocation ? SOS_E_NOMEM : SOS_E_CUDA;
}

// C(a, b) for the small arguments of this library (results fit in int64).
static int64_t binom(int64_t a, int64_t b) {
    if (b < 0 || a < b) return 0;
    b = std::min(b, a - b);
    __int128 v = 1;
    for (int64_t i = 1; i <= b; ++i) v = v * (a - b + i) / i;
    if (v > INT64_MAX) return -1;
    return (int64_t)v;
}

// Appends every tuple of total degree exactly D, lexicographically descending.
static void gen_degree(int n, int i, int remaining, uint8_t* cur, std::vector<uint8_t>& out) {
    if (i == n - 1) {
        cur[i] = (uint8_t)remaining;
        out.insert(out.end(), cur, cur + n);
        return;
    }
    for (int e = remaining; e >= 0; --e) {
        cur[i] = (uint8_t)e;
        gen_degree(n, i + 1, remaining - e, cur, out);
    }
}

static std::vector<uint8_t> gen_table(int n, int deg) {
    std::vector<uint8_t> out;
    std::vector<uint8_t> cur(n);
    for (int D = deg; D >= 0; --D) gen_degree(n, 0, D, cur.data(), out);
    return out;
}

Workspace workspace_layout(const sos_plan_s* p, int prec) {
    Workspace w;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (bytes + 255) / 256 * 256;
        return at;
    };
    const size_t elt = (prec == SOS_FP64 || prec == SOS_FP64_TC) ? 8 : 4;
    w.status = take(64 * sizeof(int32_t));
    w.partials = take(2 * kResidBlocks * sizeof(double));
    w.loss = take(2 * sizeof(double));
    w.c = take((size_t)p->M * elt);
    w.resid = take((size_t)p->M * elt);
    w.grad = take((size_t)p->N * (size_t)p->r * (prec == SOS_FP64_TC ? 4 : elt));
    if (prec == SOS_BF16) {
        w.a16 = take(2 * (size_t)p->N * (size_t)p->ld16 * 2);
        w.diag = take((size_t)p->N * sizeof(float));
        if (use_h_ring()) {
            const RingGeometry g = ring_geometry(p);
            w.ring = take((size_t)g.slots * 256 * (size_t)p->ld16h * 2);
            w.ring_flags = take(((size_t)64 + 2 * (size_t)g.panels) * sizeof(uint32_t));
        } else {
            w.h16 = take((size_t)p->N * (size_t)p->ld16h * 2);
        }
    }
    if (prec == SOS_FP64_TC) {
        w.a16 = take((size_t)p->N * (size_t)p->ld16 * 2);
        w.h16 = take((size_t)p->N * (size_t)p->ld16h * 2);
        w.resid32 = take((size_t)p->M * 4);
        const SliceFormat f = slice_format(p);
        w.slices = take((size_t)f.max_slices * (size_t)round_up(p->N, 256) * (size_t)f.ld * f.elem_bytes);
        w.ex = take((size_t)p->N * 4);
    }
    w.total = off;
    return w;
}

}  // namespace sos

using namespace sos;

extern "C" {

const char* sos_last_error(void) { return g_last_error.c_str(); }

int sos_plan_create(int n, int two_d, int64_t r, sos_plan_t* out) {
    if (!out) return fail(SOS_E_INVALID, "sos_plan_create: out is NULL");
    *out = nullptr;
    if (n < 1 || two_d < 2 || (two_d & 1) || r < 1 || n + two_d > 255)
        return fail(SOS_E_INVALID, "sos_plan_create: need n >= 1, even two_d >= 2, r >= 1, n + two_d <= 255");
    const int d = two_d / 2;
    const int64_t N = binom(n + d, d), M = binom(n + two_d, two_d);
    if (N <= 0 || M <= 0 || M >= (int64_t(1) << 31))
        return fail(SOS_E_NOMEM, "sos_plan_create: more than 2^31 coefficients");
    sos_plan_s* p = new (std::nothrow) sos_plan_s();
    if (!p) return fail(SOS_E_NOMEM, "sos_plan_create: out of host memory");
    try {
        p->n = n;
        p->two_d = two_d;
        p->d = d;
        p->N = N;
        p->M = M;
        p->r = r;
        p->ld_idx = round_up(N, 8);
        p->ld16 = round_up(r, 64);
        p->ld16h = round_up(N, 64);
        p->Ed = gen_table(n, d);
        p->E2d = gen_table(n, two_d);
        if ((int64_t)p->Ed.size() != N * n || (int64_t)p->E2d.size() != M * n) {
            delete p;
            return fail(SOS_E_INVALID, "sos_plan_create: internal table size mismatch");
        }
        // suffix sums S_j(a), j = 0..n-1 (0-based), for the rows of Ed
        p->Sd.resize((size_t)N * n);
        for (int64_t a = 0; a < N; ++a) {
            int s = 0;
            for (int j = n - 1; j >= 0; --j) {
                s += p->Ed[a * n + j];
                p->Sd[a * n + j] = (uint8_t)s;
            }
        }
        // phi[j][s] for 0-based j: j = 0 covers the higher-degree blocks,
        // j >= 1 the tuples of the same degree that are larger at position j-1.
        const int W = two_d + 1;
        p->phi.assign((size_t)n * W, 0);
        for (int s = 0; s <= two_d; ++s) {
            int64_t acc = 0;
            for (int t = s + 1; t <= two_d; ++t) acc += binom(t + n - 1, n - 1);
            p->phi[s] = (int32_t)acc;
        }
        for (int j = 1; j < n; ++j)        // 1-based position j+1
            for (int s = 1; s <= two_d; ++s)
                p->phi[(size_t)j * W + s] = (int32_t)binom(s + n - (j + 1), n - (j + 1) + 1);
    } catch (const std::bad_alloc&) {
        delete p;
        return fail(SOS_E_NOMEM, "sos_plan_create: out of host memory");
    }
    *out = p;
    return SOS_OK;
}

int sos_plan(int n, int two_d, int64_t r, sos_plan_t* out) { return sos_plan_create(n, two_d, r, out); }

int sos_plan_destroy(sos_plan_t p) {
    if (!p) return SOS_OK;
    if (p->dev.device >= 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(p->dev.device);
        cudaFree(p->dev.idx);
        cudaFree(p->dev.fwd_tiles);
        cudaFree(p->dev.adj_tiles);
        cudaFree(p->dev.fwd_tiles2);
        cudaFree(p->dev.adj_tiles2);
        cudaFree(p->dev.panel_tiles);
        cudaFree(p->dev.fwd_units);
        cudaFree(p->dev.adj_units);
        cudaFree(p->dev.pair_ptr);
        cudaFree(p->dev.pair_pos);
        cudaFree(p->dev.form_rows);
        cudaFree(p->dev.form_pairs);
        cudaFree(p->dev.slice_tiles2);
        cudaFree(p->dev.slice_groups);
        if (cur >= 0) cudaSetDevice(cur);
    }
    delete p;
    return SOS_OK;
}

int sos_plan_sizes(sos_plan_t p, int64_t* N, int64_t* M, int64_t* r) {
    if (!p) return fail(SOS_E_INVALID, "sos_plan_sizes: NULL plan");
    if (N) *N = p->N;
    if (M) *M = p->M;
    if (r) *r = p->r;
    return SOS_OK;
}

int sos_plan_monomials(sos_plan_t p, int which, uint8_t* exps) {
    if (!p || !exps || (which != 0 && which != 1))
        return fail(SOS_E_INVALID, "sos_plan_monomials: bad argument");
    const auto& t = which == 0 ? p->Ed : p->E2d;
    std::memcpy(exps, t.data(), t.size());
    return SOS_OK;
}

int sos_plan_idx(sos_plan_t p, int32_t* idx) {
    if (!p || !idx) return fail(SOS_E_INVALID, "sos_plan_idx: bad argument");
    if (p->N * p->N > (int64_t(1) << 31)) return fail(SOS_E_NOMEM, "sos_plan_idx: table too large");
    const int n = p->n, W = p->two_d + 1;
    const int64_t N = p->N;
    for (int64_t a = 0; a < N; ++a) {
        const uint8_t* Sa = &p->Sd[a * n];
        for (int64_t b = 0; b < N; ++b) {
            const uint8_t* Sb = &p->Sd[b * n];
            int32_t g = 0;
            for (int j = 0; j < n; ++j) g += p->phi[(size_t)j * W + Sa[j] + Sb[j]];
            idx[a * N + b] = g;
        }
    }
    return SOS_OK;
}

int sos_plan_device_idx(sos_plan_t p, int64_t row0, int64_t rows, int32_t* idx) {
    if (!p || !idx || row0 < 0 || rows < 0 || row0 + rows > p->N)
        return fail(SOS_E_INVALID, "sos_plan_device_idx: bad argument");
    SOS_CHECK(ensure_device(p));
    if (rows == 0) return SOS_OK;
    const size_t row_bytes = (size_t)p->N * sizeof(int32_t);
    SOS_CUDA(cudaMemcpy2D(idx, row_bytes, p->dev.idx + row0 * p->ld_idx, (size_t)p->ld_idx * sizeof(int32_t),
                          row_bytes, (size_t)rows, cudaMemcpyDeviceToHost));
    return SOS_OK;
}

int sos_workspace_size(sos_plan_t p, int prec, size_t* bytes) {
    if (!p || !bytes || prec < SOS_BF16 || prec > SOS_FP64_TC)
        return fail(SOS_E_INVALID, "sos_workspace_size: bad argument");
    *bytes = workspace_layout(p, prec).total;
    return SOS_OK;
}

}  // extern "C"

namespace sos {

// Tile lists.  The forward computes the upper triangle of A A^T in tiles of
// 128 rows (I) x 256 columns (J); a tile is needed when it holds some b >= a,
// i.e. J >= floor(I / 2).  The adjoint covers N x r in tiles of 128 x 256.
// Both lists walk bands of row blocks so that the CTAs running at the same
// time share operand panels in L2.
// Units of two tiles sharing the column block y: consecutive row blocks of
// `rows` pair up; an odd one out gets a stand-in (x = -1 - x) that recomputes
// it and stores nothing.
static void push_units(std::vector<int2>& out, const std::vector<int>& rows, int y) {
    for (size_t k = 0; k < rows.size(); k += 2) {
        out.push_back(make_int2(rows[k], y));
        out.push_back(k + 1 < rows.size() ? make_int2(rows[k + 1], y) : make_int2(-1 - rows[k], y));
    }
}

static void make_units(const sos_plan_s* p, std::vector<int2>& fwd_u, std::vector<int2>& adj_u) {
    const int TP = (int)ceil_div(p->N, 256), TK = (int)ceil_div(p->r, 256);
    const int bf = 8, ba = adjoint_band();
    std::vector<int> rows;
    for (int i0 = 0; i0 < TP; i0 += bf) {
        const int i1 = std::min(TP, i0 + bf);
        for (int J = i0; J < TP; ++J) {
            rows.clear();
            for (int I = i0; I < i1; ++I)
                if (J >= I) rows.push_back(I);
            push_units(fwd_u, rows, J);
        }
    }
    for (int i0 = 0; i0 < TP; i0 += ba) {
        const int i1 = std::min(TP, i0 + ba);
        for (int K = 0; K < TK; ++K) {
            rows.clear();
            for (int I = i0; I < i1; ++I) rows.push_back(I);
            push_units(adj_u, rows, K);
        }
    }
}

static void make_tiles(const sos_plan_s* p, int pairs, std::vector<int2>& fwd, std::vector<int2>& adj,
                       std::vector<int2>& fwd2, std::vector<int2>& adj2) {
    const int TI = (int)ceil_div(p->N, 128), TJ = (int)ceil_div(p->N, 256);
    const int band = 16;
    for (int i0 = 0; i0 < TI; i0 += band) {
        const int i1 = std::min(TI, i0 + band);
        for (int J = i0 / 2; J < TJ; ++J)
            for (int I = i0; I < i1; ++I)
                if (J >= I / 2) fwd.push_back(make_int2(I, J));
    }
    const int TK = (int)ceil_div(p->r, 256);
    for (int i0 = 0; i0 < TI; i0 += band) {
        const int i1 = std::min(TI, i0 + band);
        for (int K = 0; K < TK; ++K)
            for (int I = i0; I < i1; ++I) adj.push_back(make_int2(I, K));
    }
    // 256 x 256 tiles for CTA pairs: upper triangle J >= I for the forward.
    // Both lists walk bands of row blocks (rows fastest inside a band) so the
    // pairs running at once share operand panels in L2; the band heights can
    // be overridden with SOS_BAND_FWD / SOS_BAND_ADJ (tuning).
    const int TP = (int)ceil_div(p->N, 256);
    auto env_band = [](const char* name, int dflt) {
        const char* e = std::getenv(name);
        const int v = e ? std::atoi(e) : 0;
        return v > 0 ? v : dflt;
    };
    const int bf = env_band("SOS_BAND_FWD", 8), ba = adjoint_band();
    for (int i0 = 0; i0 < TP; i0 += bf) {
        const int i1 = std::min(TP, i0 + bf);
        for (int J = i0; J < TP; ++J)
            for (int I = i0; I < i1; ++I)
                if (J >= I) fwd2.push_back(make_int2(I, J));
    }
    for (int i0 = 0; i0 < TP; i0 += ba) {
        const int i1 = std::min(TP, i0 + ba);
        for (int K = 0; K < TK; ++K)
            for (int I = i0; I < i1; ++I) adj2.push_back(make_int2(I, K));
    }
    // The persistent adjoint gives tile t to pair t mod `pairs`, so a list of
    // T tiles takes ceil(T / pairs) rounds, the last holding R = T mod pairs
    // tiles.  When R <= pairs / 2, those R tiles become narrow 128-column
    // halves (one half when the tile's valid width is at most 128); the last
    // round then runs at most 2R half tiles on as many pairs and takes half
    // as long.
    const int T = (int)adj2.size();
    const int R = pairs > 0 ? T % pairs : 0;
    if (R > 0 && 2 * R <= pairs) {
        std::vector<int2> tail(adj2.end() - R, adj2.end());
        adj2.resize(T - R);
        for (const int2& tl : tail) {
            const int64_t w = std::min<int64_t>(256, p->r - (int64_t)tl.y * 256);
            adj2.push_back(make_int2(tl.x, -(2 * tl.y + 1)));
            if (w > 128) adj2.push_back(make_int2(tl.x, -(2 * tl.y + 2)));
        }
    }
}

int adjoint_band() {
    static const int v = [] {
        const char* e = std::getenv("SOS_BAND_ADJ");
        const int b = e ? std::atoi(e) : 0;
        return b > 0 ? b : 8;
    }();
    return v;
}

bool use_mcast() {
    static const bool v = [] {
        const char* e = std::getenv("SOS_MCAST");
        return e && e[0] == '1';
    }();
    return v && use_cta_pairs() && !use_h_ring();
}

bool use_exact_diag() {
    static const bool v = [] {
        const char* e = std::getenv("SOS_EXACT_DIAG");
        return e && e[0] == '1';
    }();
    return v;
}

int slice_fp8_setting() {
    static const int v = [] {
        const char* e = std::getenv("SOS_SLICE_FP8");
        if (!e || !e[0]) return -1;
        return e[0] == '1' ? 1 : 0;
    }();
    return v;
}

SliceFormat slice_format(const sos_plan_s* p) {
    SliceFormat f;
    const int want = slice_fp8_setting();
    const bool bf16_exact = p->r * 31 * 31 < ((int64_t)1 << 24);
    if (want == 1 || (want < 0 && !bf16_exact)) {
        f.fp8 = true;
        f.bits = 4;
        f.dmax = 15;
        f.max_slices = kMaxSlices8;
        f.ld = round_up(p->r, 16);      // bytes: TMA wants 16-byte row strides
        f.elem_bytes = 1;
    } else {
        f.ld = p->ld16;
    }
    return f;
}

bool use_h_ring() {
    static const bool v = [] {
        const char* e = std::getenv("SOS_H_RING");
        return e && e[0] == '1';
    }();
    return v && use_cta_pairs();
}

// Slots of the ring in bands (SOS_RING_DEPTH, default 3, at least 2): with
// depth D, the builders of band b + D - 1 need only band b - 1 to be done.
static int ring_depth() {
    static const int v = [] {
        const char* e = std::getenv("SOS_RING_DEPTH");
        const int d = e ? std::atoi(e) : 0;
        return d >= 2 ? d : 3;
    }();
    return v;
}

RingGeometry ring_geometry(const sos_plan_s* p) {
    RingGeometry g;
    g.panels = (int)ceil_div(p->N, 256);
    g.band = std::min(adjoint_band(), g.panels);
    g.slots = std::min(ring_depth() * g.band, g.panels);
    return g;
}

bool use_cta_pairs() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("SOS_CTA_PAIRS");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

int ensure_device(sos_plan_s* p) {
    std::lock_guard<std::mutex> lock(p->mu);
    int cur = -1;
    SOS_CUDA(cudaGetDevice(&cur));
    if (p->dev.device == cur) return SOS_OK;
    if (p->dev.device >= 0)
        return fail(SOS_E_INVALID, "plan already resident on another device");
    DeviceTables t;
    t.device = cur;
    SOS_CUDA(cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, cur));
    const size_t idx_bytes = (size_t)p->N * (size_t)p->ld_idx * sizeof(int32_t);
    std::vector<int2> fwd, adj, fwd2, adj2;
    int pairs = 0;
    if (use_cta_pairs()) SOS_CHECK(adjoint_pair_capacity(&pairs));
    make_tiles(p, pairs, fwd, adj, fwd2, adj2);
    // adjoint tiles per 256-row panel (the ring's slot-release counts)
    std::vector<int32_t> panel_tiles((size_t)ceil_div(p->N, 256), 0);
    for (const int2& tl : adj2) panel_tiles[tl.x]++;
    std::vector<int2> fwd_u, adj_u;
    if (use_mcast()) make_units(p, fwd_u, adj_u);
    uint8_t* d_S = nullptr;
    int32_t* d_phi = nullptr;
    cudaError_t e = cudaMalloc(&t.idx, idx_bytes);
    if (e == cudaSuccess && !fwd_u.empty()) e = cudaMalloc(&t.fwd_units, fwd_u.size() * sizeof(int2));
    if (e == cudaSuccess && !adj_u.empty()) e = cudaMalloc(&t.adj_units, adj_u.size() * sizeof(int2));
    if (e == cudaSuccess && !fwd_u.empty())
        e = cudaMemcpy(t.fwd_units, fwd_u.data(), fwd_u.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !adj_u.empty())
        e = cudaMemcpy(t.adj_units, adj_u.data(), adj_u.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t.panel_tiles, panel_tiles.size() * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(t.panel_tiles, panel_tiles.data(), panel_tiles.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t.fwd_tiles, fwd.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&t.adj_tiles, adj.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&t.fwd_tiles2, fwd2.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&t.adj_tiles2, adj2.size() * sizeof(int2));
    if (e == cudaSuccess)
        e = cudaMemcpy(t.fwd_tiles2, fwd2.data(), fwd2.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t.adj_tiles2, adj2.data(), adj2.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&d_S, p->Sd.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_phi, p->phi.size() * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(t.fwd_tiles, fwd.data(), fwd.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t.adj_tiles, adj.data(), adj.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_S, p->Sd.data(), p->Sd.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_phi, p->phi.data(), p->phi.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    int rc = SOS_OK;
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "ensure_device: upload");
    } else {
        rc = launch_build_idx(p, t.idx, d_S, d_phi, 0);
        if (rc == SOS_OK) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) rc = cuda_fail(e, "ensure_device: build idx");
        }
    }
    cudaFree(d_S);
    cudaFree(d_phi);
    if (rc != SOS_OK) {
        cudaFree(t.idx);
        cudaFree(t.fwd_tiles);
        cudaFree(t.adj_tiles);
        cudaFree(t.fwd_tiles2);
        cudaFree(t.adj_tiles2);
        cudaFree(t.panel_tiles);
        cudaFree(t.fwd_units);
        cudaFree(t.adj_units);
        return rc;
    }
    t.num_fwd_tiles = (int)fwd.size();
    t.num_adj_tiles = (int)adj.size();
    t.num_fwd_tiles2 = (int)fwd2.size();
    t.num_adj_tiles2 = (int)adj2.size();
    t.num_fwd_units = (int)(fwd_u.size() / 2);
    t.num_adj_units = (int)(adj_u.size() / 2);
    p->dev = t;
    return SOS_OK;
}

}  // namespace sos

namespace sos {

// Pair lists for gathering c_g = sum over pairs (a <= b, a + b = g) of
// w_ab G_ab without atomics: a counting sort of the upper triangle of the
// index table by coefficient.
int ensure_pair_lists(sos_plan_s* p) {
    SOS_CHECK(ensure_device(p));
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->dev.pair_ptr) return SOS_OK;
    if (p->N > 46340) return fail(SOS_E_UNSUPPORTED, "pair lists: N too large for 32-bit positions");
    const int n = p->n, W = p->two_d + 1;
    const int64_t N = p->N, M = p->M;
    std::vector<int32_t> ptr(M + 1, 0);
    auto rank = [&](int64_t a, int64_t b) {
        int32_t g = 0;
        for (int j = 0; j < n; ++j) g += p->phi[(size_t)j * W + p->Sd[a * n + j] + p->Sd[b * n + j]];
        return g;
    };
    for (int64_t a = 0; a < N; ++a)
        for (int64_t b = a; b < N; ++b) ptr[rank(a, b) + 1]++;
    for (int64_t g = 0; g < M; ++g) ptr[g + 1] += ptr[g];
    std::vector<int32_t> pos(ptr[M]);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t a = 0; a < N; ++a)
        for (int64_t b = a; b < N; ++b) {
            const int32_t g = rank(a, b);
            int32_t v = (int32_t)(a * N + b);
            if (a == b) v |= INT32_MIN;
            pos[fill[g]++] = v;
        }
    int32_t *d_ptr = nullptr, *d_pos = nullptr;
    cudaError_t e = cudaMalloc(&d_ptr, ptr.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_pos, std::max<size_t>(1, pos.size()) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_ptr, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_pos, pos.data(), pos.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_ptr);
        cudaFree(d_pos);
        return cuda_fail(e, "pair lists: upload");
    }
    p->dev.pair_ptr = d_ptr;
    p->dev.pair_pos = d_pos;
    return SOS_OK;
}

}  // namespace sos
