// C ABI of libnqs_sr: argument checks, workspace carving and the order of the
// stages of one block-layer SR step (see include/nqs_sr.h for the contract).
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <new>
#include <atomic>
#include <mutex>
#include <cuda_bf16.h>
#include "internal.cuh"
#include "eigh.cuh"

using namespace nqs;

static std::atomic<int> g_dp_fallback_all{0};
bool nqs::dp_fallback_all() { return g_dp_fallback_all.load() != 0; }

constexpr int NSTAGE = 6;  // jacobian, local energy, centring+force, gram, tridiagonal reduction, solve
struct nqs_workspace {
    char* base;
    size_t bytes;
    bool timing;
    bool recorded;
    cudaEvent_t ev[NSTAGE + 1];
};

unsigned long long& nqs::launch_counter() {
    static unsigned long long n = 0;
    return n;
}

namespace {
constexpr int QL_MAXIT_DEFAULT = 60;
constexpr int REF_MAXIT_DEFAULT = 30;
constexpr unsigned long long WAIT_NS_DEFAULT = 2000000000ull;
std::atomic<int> g_ql_maxit{QL_MAXIT_DEFAULT};
std::atomic<int> g_ref_maxit{REF_MAXIT_DEFAULT};
std::atomic<unsigned long long> g_wait_ns{WAIT_NS_DEFAULT};
}  // namespace

namespace {
constexpr int GRAM_TUNE_MAX = 64;
struct GramTune {
    long long max_nb, max_ns;
    int group;
};
std::mutex g_tune_mu;
int g_tune_n = 0;
GramTune g_tune[GRAM_TUNE_MAX];
}  // namespace

int nqs::gram_group_edge(long long max_nb, long long ns) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int i = 0; i < g_tune_n; ++i)
        if (max_nb <= g_tune[i].max_nb && ns <= g_tune[i].max_ns) return g_tune[i].group;
    return GRAM_GROUP_EDGE_DEFAULT;
}

nqs::Limits nqs::limits() {
    return Limits{g_ql_maxit.load(std::memory_order_relaxed), g_ref_maxit.load(std::memory_order_relaxed),
                  g_wait_ns.load(std::memory_order_relaxed)};
}

namespace {

thread_local std::string g_err = "";

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(NQS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(expr, where)                               \
    do {                                              \
        cudaError_t _e = (expr);                      \
        if (_e != cudaSuccess) return cuda_fail(_e, where); \
    } while (0)

constexpr size_t STATUS_BYTES = 256;
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bump allocator over the caller's workspace (after the status header).
struct Arena {
    char* base;
    size_t cap, used;
    void* take(size_t bytes) {
        void* p = base ? base + used : nullptr;
        used += al256(bytes);
        return p;
    }
};
Arena arena_of(nqs_workspace* ws) {
    Arena a;
    a.base = ws ? ws->base + STATUS_BYTES : nullptr;
    a.cap = ws ? (ws->bytes > STATUS_BYTES ? ws->bytes - STATUS_BYTES : 0) : 0;
    a.used = 0;
    return a;
}
Arena sizing_arena() { return Arena{nullptr, 0, 0}; }

DevStatus* status_of(nqs_workspace* ws) { return reinterpret_cast<DevStatus*>(ws->base); }

// O (and the Jacobian arithmetic) is FP64 except in NQS_FP32 mode
inline size_t csize(int prec) { return prec == NQS_FP32 ? sizeof(c64) : sizeof(c128); }
inline int jac_prec(int prec) { return prec == NQS_FP32 ? NQS_FP32 : NQS_FP64; }
// local energies: FP32 arithmetic only in NQS_FP32 mode (in the split modes an FP32
// E_loc alone moves dtheta by ~1e-5 relative on the 10x10 workload)
inline int eloc_prec(int prec) { return prec == NQS_FP32 ? NQS_FP32 : NQS_FP64; }
// NQS_ELOC_DIFF32: FFNN local energies by FP32 difference propagation (the FP64-class
// double-float kernel for the connections it cannot follow); needs the FP64 forward of the
// parents, i.e. any precision but NQS_FP32
inline bool eloc_dp(int prec, int flags) { return (flags & NQS_ELOC_DIFF32) && prec != NQS_FP32; }
inline int nsplit_of(int prec) {
    return prec == NQS_SPLIT_BF16 ? 2 : (prec == NQS_SPLIT_BF16X3 ? 3 : (prec == NQS_SPLIT_BF16_EXACT ? 5 : 0));
}
// Refinement target of the Cholesky solve inside a step: 1e-14 ||F||, or 1e-12 ||F|| when S comes
// from a split Gram (whose own entry error is ~1e-10 relative); the solution error is then at
// most 1e-12 kappa(S~) relative (1.4e-8 for kappa 1.4e4), far below the split's dtheta bar.
inline double step_ref_tol(int prec) { return nsplit_of(prec) ? 1e-12 : 1e-14; }
inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

int check_prec(int prec) {
    if (prec != NQS_FP64 && prec != NQS_FP32 && prec != NQS_SPLIT_BF16 && prec != NQS_SPLIT_BF16X3 &&
        prec != NQS_SPLIT_BF16_EXACT)
        return fail(NQS_ERR_INVALID_ARG, "unknown precision %d", prec);
    return NQS_OK;
}

int check_offsets(const int64_t* off, int nb, long long np) {
    if (!off || nb < 1) return fail(NQS_ERR_INVALID_ARG, "block_off is NULL or n_blocks < 1");
    if (nb > MAXB) return fail(NQS_ERR_INVALID_ARG, "n_blocks %d exceeds the limit %d", nb, MAXB);
    if (off[0] != 0) return fail(NQS_ERR_INVALID_ARG, "block_off[0] must be 0");
    for (int b = 0; b < nb; ++b)
        if (off[b + 1] <= off[b]) return fail(NQS_ERR_INVALID_ARG, "block_off not strictly increasing at %d", b);
    if (np >= 0 && off[nb] != np)
        return fail(NQS_ERR_INVALID_ARG, "block_off[n_blocks] = %lld != n_p = %lld", (long long)off[nb], np);
    return NQS_OK;
}

int ham_desc(const nqs_hamiltonian* h, int n_sites, HamDesc* hd) {
    if (!h || !h->bond_ij || !h->bond_J) return fail(NQS_ERR_INVALID_ARG, "hamiltonian or bond arrays NULL");
    if (h->n_sites != n_sites) return fail(NQS_ERR_INVALID_ARG, "hamiltonian has %d sites, model %d", h->n_sites, n_sites);
    if (h->n_bonds < 1 || h->n_bonds > 16 * MAXN) return fail(NQS_ERR_INVALID_ARG, "bad n_bonds %d", h->n_bonds);
    if (h->sign_rule != 1 && h->sign_rule != -1) return fail(NQS_ERR_INVALID_ARG, "sign_rule must be +-1");
    hd->n_sites = h->n_sites;
    hd->n_bonds = h->n_bonds;
    hd->bond_ij = h->bond_ij;
    hd->bond_J = h->bond_J;
    hd->c = h->c;
    hd->sign_rule = h->sign_rule;
    return NQS_OK;
}

// ------------------------------------------------------------------ stage plans
struct JacBufs {
    void *thR, *wtR, *Z, *G;
    c128* logpsi;
};
void plan_model(Arena& a, const ModelDesc& md, long long ns, int prec, JacBufs* b, bool need_G) {
    const size_t cs = csize(prec);
    b->thR = a.take(cs * md.n_p);
    b->wtR = a.take(cs * (size_t)(model_wt_elems(md) > 0 ? model_wt_elems(md) : 1));
    b->Z = a.take(cs * (size_t)model_z_elems(md, ns));
    b->G = need_G ? a.take(cs * (size_t)model_z_elems(md, ns)) : nullptr;
    b->logpsi = static_cast<c128*>(a.take(sizeof(c128) * ns));
}

struct ElocBufs {
    int32_t *cnt, *cbond, *csamp;
    long long* off;
    c128* terms;
    void* wdf;  // double-float (hi, lo) copy of the transposed weights (FP64 local energies)
    DpBufs dp;  // FP32 difference propagation (FFNN models only; null otherwise)
};
void plan_eloc(Arena& a, const ModelDesc& md, long long ns, int nbonds, ElocBufs* b) {
    const long long we = model_wt_elems(md);
    b->wdf = a.take(16 * (size_t)(we > 0 ? we : 1));
    const long long maxc = ns * nbonds;
    b->cnt = static_cast<int32_t*>(a.take(4 * ns));
    b->off = static_cast<long long*>(a.take(8 * (ns + 1)));
    b->cbond = static_cast<int32_t*>(a.take(4 * maxc));
    b->csamp = static_cast<int32_t*>(a.take(4 * maxc));
    b->terms = static_cast<c128*>(a.take(16 * maxc));
    b->dp = DpBufs{nullptr, nullptr, nullptr, nullptr};
    if (dp_applicable(md)) {
        b->dp.w32 = static_cast<float2*>(a.take(8 * (size_t)(we > 0 ? we : 1)));
        b->dp.pz = static_cast<float4*>(a.take(16 * (size_t)model_z_elems(md, ns)));
        b->dp.fb_list = static_cast<long long*>(a.take(8 * (size_t)(maxc > 0 ? maxc : 1)));
        b->dp.fb_count = static_cast<unsigned long long*>(a.take(8));
    }
}

struct BuildBufs {
    c128* e;
    c128* means;  // global means of a sample-sharded step (n_p + 1)
    void* planes[5];
    double* diag;
    int8_t* gexp;
    long long ldk;
};
void plan_build(Arena& a, long long ns, long long np, int prec, BuildBufs* b) {
    b->e = static_cast<c128*>(a.take(16 * ns));
    b->means = static_cast<c128*>(a.take(16 * (np + 1)));
    b->ldk = round_up(ns, 64);
    const int nsp = nsplit_of(prec);
    for (int i = 0; i < 5; ++i)
        b->planes[i] = i < plane_units(nsp) ? a.take(2ull * 2 * np * plane_row_len(nsp, i, b->ldk)) : nullptr;
    b->diag = nsp ? static_cast<double*>(a.take(8 * np)) : nullptr;
    b->gexp = nsp == 5 ? static_cast<int8_t*>(a.take((size_t)(b->ldk / GRAM_GROUP) * np)) : nullptr;
}

// ------------------------------------------------------------------ stages
int run_model(const ModelDesc& md, int prec, const void* theta, const int8_t* x, long long ns,
              const JacBufs& b, cudaStream_t st) {
    CK(launch_prepare_params(prec, md, theta, b.thR, b.wtR, st), "prepare_params");
    CK(launch_forward(prec, md, b.thR, b.wtR, x, ns, b.Z, b.logpsi, st), "forward");
    return NQS_OK;
}

int run_eloc(const ModelDesc& md, int prec, const HamDesc& hd, const int8_t* x, long long ns,
             const JacBufs& jb, const ElocBufs& eb, c128* eloc, DevStatus* status, cudaStream_t st,
             bool dp = false) {
    CK(launch_conn_count(x, ns, hd, eb.cnt, status, st), "conn_count");
    CK(launch_scan(eb.cnt, ns, eb.off, st), "scan");
    CK(launch_conn_fill(x, ns, hd, eb.off, eb.cbond, eb.csamp, st), "conn_fill");
    if (dp && prec == NQS_FP64 && eb.dp.pz) {
        CK(launch_conn_terms_dp(md, jb.thR, jb.wtR, eb.wdf, jb.Z, jb.logpsi, x, ns, hd, eb.cbond, eb.csamp,
                                eb.off + ns, ns * hd.n_bonds, eb.terms, eb.dp, st),
           "conn_terms_dp");
        CK(launch_eloc_reduce(x, ns, hd, eb.off, eb.terms, eloc, status, st), "eloc_reduce");
        return NQS_OK;
    }
    if (prec == NQS_FP64) CK(launch_split_weights(md, jb.wtR, eb.wdf, st), "split_weights");
    CK(launch_conn_terms(prec, md, jb.thR, jb.wtR, eb.wdf, jb.Z, jb.logpsi, x, hd, eb.cbond, eb.csamp, eb.off + ns,
                         ns * hd.n_bonds, eb.terms, st),
       "conn_terms");
    CK(launch_eloc_reduce(x, ns, hd, eb.off, eb.terms, eloc, status, st), "eloc_reduce");
    return NQS_OK;
}

int run_build(void* O, long long ldo, long long ns, long long np, const double* w, const int64_t* off, int nb,
              const c128* eloc, int prec, c128* S, c128* F, c128* Omean, c128* Emean, const BuildBufs& bb,
              DevStatus* status, cudaStream_t st, cudaEvent_t gram_event = nullptr) {
    CK(launch_emean(eloc, w, ns, Emean, bb.e, status, st), "emean");
    const int nsp = nsplit_of(prec);
    CK(launch_center(prec, nsp, O, ldo, ns, np, w, bb.e, F, Omean, nsp ? bb.planes : nullptr, bb.ldk, bb.diag,
                     bb.gexp, np, status, st),
       "center");
    if (gram_event) CK(cudaEventRecord(gram_event, st), "event");
    GramTable* tab = new (std::nothrow) GramTable;
    if (!tab) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
    const double scale = w ? 1.0 : 1.0 / (double)ns;
    cudaError_t e;
    if (nsp) {
        gram_table(off, nb, 64, tab);
        e = launch_gram_tc(nsp, bb.planes, bb.gexp, np, 2 * np, bb.ldk, bb.ldk, scale, *tab, S, status, st);
        // the diagonal (sum_s w_s |dO_k|^2) is taken from the FP64 centring pass
        if (e == cudaSuccess) e = launch_set_diag(S, *tab, bb.diag, st);
    } else {
        gram_table(off, nb, 64, tab);
        e = launch_gram_simt(prec, O, ldo, ns, w, scale, *tab, S, st);
    }
    delete tab;
    if (e == cudaErrorNotSupported) return fail(NQS_ERR_UNSUPPORTED, "tensor-core Gram needs an sm_103 device");
    CK(e, "gram");
    return NQS_OK;
}

int run_solve(c128* S, const int64_t* off, int nb, const c128* F, double shift, double cutoff, int mode,
              double eta, int solver, c128* dtheta, double* evals, int32_t* n_kept, Arena& a, DevStatus* status,
              cudaStream_t st, cudaEvent_t trd_event = nullptr, cudaEvent_t trd_start = nullptr,
              bool graph = false, double ref_tol = 1e-14) {
    if (solver != NQS_SOLVE_FP64 && solver != NQS_SOLVE_MIXED && solver != NQS_SOLVE_MIXED_PSD)
        return fail(NQS_ERR_INVALID_ARG, "unknown solver %d", solver);
    if (!(shift >= 0.0)) return fail(NQS_ERR_INVALID_ARG, "diag_shift must be >= 0");
    if (!(cutoff >= 0.0)) return fail(NQS_ERR_INVALID_ARG, "cutoff must be >= 0");
    if (mode != 0 && mode != 1) return fail(NQS_ERR_INVALID_ARG, "cutoff_mode must be 0 or 1");
    const size_t need = solve_workspace_bytes(off, nb);
    void* work = a.take(need);
    SolveArgs sa{shift, cutoff, eta, mode, evals != nullptr, solver != NQS_SOLVE_FP64, solver == NQS_SOLVE_MIXED_PSD,
                 trd_event, trd_start, graph, limits().ql_maxit};
    sa.ref_tol = ref_tol;
    const int rc = launch_block_solve(S, off, nb, F, sa, dtheta, evals, n_kept, work, need, status, st);
    if (rc == NQS_ERR_UNSUPPORTED) return fail(rc, "block larger than the solver limit");
    if (rc != NQS_OK) return fail(rc, "block solve launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return NQS_OK;
}

// exchange-move sampler: FP64 forward of the chains, the proposals as a bond table, the
// FP64 connected forwards' ratios
struct McBufs {
    JacBufs jb;
    void* wdf;
    int32_t *pairs, *valid, *csamp, *cbond;
    double* bond_J;
    long long* nconn;
    c128* ratio;
};
void plan_mc(Arena& a, const ModelDesc& md, long long n, McBufs* b) {
    plan_model(a, md, n, NQS_FP64, &b->jb, false);
    const long long we = model_wt_elems(md);
    b->wdf = a.take(16 * (size_t)(we > 0 ? we : 1));
    b->pairs = static_cast<int32_t*>(a.take(8 * (size_t)n));
    b->valid = static_cast<int32_t*>(a.take(4 * (size_t)n));
    b->csamp = static_cast<int32_t*>(a.take(4 * (size_t)n));
    b->cbond = static_cast<int32_t*>(a.take(4 * (size_t)n));
    b->bond_J = static_cast<double*>(a.take(8 * (size_t)n));
    b->nconn = static_cast<long long*>(a.take(8));
    b->ratio = static_cast<c128*>(a.take(16 * (size_t)n));
}

int check_ws(nqs_workspace* ws, const Arena& need) {
    if (!ws) return fail(NQS_ERR_INVALID_ARG, "workspace is NULL");
    const size_t total = need.used + STATUS_BYTES;
    if (ws->bytes < total)
        return fail(NQS_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", ws->bytes, total);
    return NQS_OK;
}

}  // namespace

// ---------------------------------------------------------------- blocks wider than the sample count
// A block with more parameters than samples (n_b > N_s) is solved in sample space by the
// push-through identity:
//   dtheta_b = -eta X_b^H pinv(X_b X_b^H + lambda I) eps,  X_b = dO_b / sqrt(N_s), eps = e / sqrt(N_s),
// an N_s x N_s problem in place of the n_b x n_b one. With lambda > 0 and the same threshold it
// equals the block's pseudo-inverse update: F_b = X_b^H eps lies in the range of S_b, on which
// S_b + lambda I and X_b X_b^H + lambda I have the same eigenvalues (the others equal lambda and
// meet no component of F_b). The narrow blocks keep the parameter-space Gram and solve.
namespace {

struct WidePlan {
    int nnar, nwide;
    int nar[MAXB], wid[MAXB];   // block indices in the caller's order
    int64_t nar_off[MAXB + 1];  // compact offsets of the narrow blocks
    long long nar_np;           // parameters in narrow blocks
    long long max_wide;         // largest wide block
};

bool is_wide(long long n, long long ns, double shift, int prec, int solver, int flags) {
    return n > ns && shift > 0.0 && solver != NQS_SOLVE_FP64 && prec != NQS_FP32 && prec != NQS_SPLIT_BF16 &&
           prec != NQS_SPLIT_BF16X3 && (flags & NQS_PARAM_SPACE) == 0;
}

void wide_plan(const int64_t* off, int nb, long long ns, double shift, int prec, int solver, int flags,
               WidePlan* wp) {
    wp->nnar = wp->nwide = 0;
    wp->nar_np = 0;
    wp->max_wide = 0;
    wp->nar_off[0] = 0;
    for (int b = 0; b < nb; ++b) {
        const long long n = off[b + 1] - off[b];
        if (is_wide(n, ns, shift, prec, solver, flags)) {
            wp->wid[wp->nwide++] = b;
            wp->max_wide = n > wp->max_wide ? n : wp->max_wide;
        } else {
            wp->nar[wp->nnar++] = b;
            wp->nar_np += n;
            wp->nar_off[wp->nnar] = wp->nar_np;
        }
    }
}

struct WideBufs {
    JacBufs jb, jbe;
    ElocBufs eb;
    void* O;
    long long ldo;
    c128 *eloc, *e, *F;
    // narrow blocks (compact)
    void* planes[5];
    double* diag;
    int8_t* gexp;
    long long ldk;
    c128 *S, *Fn, *dthn;
    int32_t* nkn;
    // wide blocks (one at a time)
    void* planesT[5];
    int8_t* gexpT;
    double* diagT;
    void* Y;
    long long ldkT, ldy;
    c128 *T, *rhs, *u;
    int32_t* keptT;
    void* solve;
    size_t solve_bytes;
};

void plan_wide(Arena& a, const ModelDesc& md, long long ns, int nbonds, const int64_t* off, int nb, int prec,
               const WidePlan& wp, WideBufs* w) {
    plan_model(a, md, ns, jac_prec(prec), &w->jb, true);
    if (eloc_prec(prec) != jac_prec(prec)) plan_model(a, md, ns, eloc_prec(prec), &w->jbe, false);
    else w->jbe = w->jb;
    plan_eloc(a, md, ns, nbonds, &w->eb);
    w->ldo = round_up(ns, 32);
    w->O = a.take(csize(prec) * (size_t)md.n_p * (size_t)w->ldo);
    w->eloc = static_cast<c128*>(a.take(16 * ns));
    w->e = static_cast<c128*>(a.take(16 * ns));
    w->F = static_cast<c128*>(a.take(16 * (size_t)md.n_p));
    const int nsp = nsplit_of(prec);
    w->ldk = round_up(ns, 64);
    const long long nn = wp.nar_np > 0 ? wp.nar_np : 1;
    for (int q = 0; q < 5; ++q)
        w->planes[q] = q < plane_units(nsp) ? a.take(2ull * 2 * nn * plane_row_len(nsp, q, w->ldk)) : nullptr;
    w->diag = nsp ? static_cast<double*>(a.take(8 * nn)) : nullptr;
    w->gexp = nsp == 5 ? static_cast<int8_t*>(a.take((size_t)(w->ldk / GRAM_GROUP) * nn)) : nullptr;
    long long sq = 0;
    for (int i = 0; i < wp.nnar; ++i) {
        const long long n = off[wp.nar[i] + 1] - off[wp.nar[i]];
        sq += n * n;
    }
    w->S = static_cast<c128*>(a.take(16 * (size_t)(sq > 0 ? sq : 1)));
    w->Fn = static_cast<c128*>(a.take(16 * nn));
    w->dthn = static_cast<c128*>(a.take(16 * nn));
    w->nkn = static_cast<int32_t*>(a.take(4 * MAXB));
    w->ldkT = round_up(wp.max_wide, 64);
    w->ldy = round_up(wp.max_wide, 32);
    for (int q = 0; q < 5; ++q)
        w->planesT[q] = q < plane_units(nsp) ? a.take(2ull * 2 * ns * plane_row_len(nsp, q, w->ldkT)) : nullptr;
    w->gexpT = nsp == 5 ? static_cast<int8_t*>(a.take((size_t)(w->ldkT / GRAM_GROUP) * ns)) : nullptr;
    w->diagT = nsp ? static_cast<double*>(a.take(8 * ns)) : nullptr;
    w->Y = nsp ? nullptr : a.take(16 * (size_t)ns * (size_t)w->ldy);
    w->T = static_cast<c128*>(a.take(16 * (size_t)ns * (size_t)ns));
    w->rhs = static_cast<c128*>(a.take(16 * ns));
    w->u = static_cast<c128*>(a.take(16 * ns));
    w->keptT = static_cast<int32_t*>(a.take(256));
    const int64_t offT[2] = {0, ns};
    size_t sb = solve_workspace_bytes(offT, 1);
    if (wp.nnar > 0) {
        const size_t sn = solve_workspace_bytes(wp.nar_off, wp.nnar);
        sb = sn > sb ? sn : sb;
    }
    w->solve_bytes = sb;
    w->solve = a.take(sb);
}

__global__ void wide_kept_kernel(const int32_t* __restrict__ keptT, long long ns, long long nb, int32_t* out) {
    // all N_s eigenvalues of X X^H + lambda I kept (the smallest equals lambda: X is centred)
    // <=> lambda kept <=> every eigenvalue of S_b + lambda I kept
    if (threadIdx.x == 0 && out) *out = keptT[0] == ns ? (int32_t)nb : keptT[0];
}

int run_step_wide(const ModelDesc& md, const HamDesc& hd, const void* theta, const int8_t* configs, long long ns,
                  const int64_t* off, int nb, double shift, double cutoff, int mode, double eta, int prec,
                  int solver, c128* dtheta, c128* Emean, int32_t* n_kept, int flags, const WidePlan& wp,
                  const WideBufs& w, nqs_workspace* ws, DevStatus* status, cudaStream_t st) {
    const int rp = jac_prec(prec), re = eloc_prec(prec);
    const bool graph = (flags & NQS_GRAPH) != 0;
    const bool tm = ws->timing && !graph;
    const int nsp = nsplit_of(prec);
    const size_t cs = csize(prec);
    if (tm) CK(cudaEventRecord(ws->ev[0], st), "event");
    int rc = run_model(md, rp, theta, configs, ns, w.jb, st);
    if (rc) return rc;
    CK(launch_backward(rp, md, w.jb.thR, w.jb.Z, ns, w.jb.G, st), "backward");
    CK(launch_jac_write(rp, md, w.jb.thR, w.jb.Z, w.jb.G, configs, ns, w.O, w.ldo, st), "jacobian");
    if (tm) CK(cudaEventRecord(ws->ev[1], st), "event");
    if (re != rp) {
        rc = run_model(md, re, theta, configs, ns, w.jbe, st);
        if (rc) return rc;
    }
    rc = run_eloc(md, re, hd, configs, ns, w.jbe, w.eb, w.eloc, status, st, eloc_dp(prec, flags));
    if (rc) return rc;
    if (tm) CK(cudaEventRecord(ws->ev[2], st), "event");
    CK(launch_emean(w.eloc, nullptr, ns, Emean, w.e, status, st), "emean");
    // centring and force: narrow blocks write their split planes (compact rows); wide blocks
    // are centred in place (FP64) for the sample-major split and the back-projection
    char* Ob = static_cast<char*>(w.O);
    for (int i = 0; i < wp.nnar; ++i) {
        const int b = wp.nar[i];
        const long long n = off[b + 1] - off[b], r0 = wp.nar_off[i];
        void* pl[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        for (int q = 0; q < plane_units(nsp); ++q)
            pl[q] = static_cast<__nv_bfloat16*>(w.planes[q]) + 2 * r0 * plane_row_len(nsp, q, w.ldk);
        CK(launch_center(prec, nsp, Ob + cs * (size_t)off[b] * (size_t)w.ldo, w.ldo, ns, n, nullptr, w.e,
                         w.F + off[b], nullptr, nsp ? pl : nullptr, w.ldk, nsp ? w.diag + r0 : nullptr,
                         nsp == 5 ? w.gexp + r0 : nullptr, wp.nar_np, status, st),
           "center");
    }
    for (int i = 0; i < wp.nwide; ++i) {
        const int b = wp.wid[i];
        CK(launch_center(NQS_FP64, 0, Ob + cs * (size_t)off[b] * (size_t)w.ldo, w.ldo, ns, off[b + 1] - off[b],
                         nullptr, w.e, w.F + off[b], nullptr, nullptr, 0, nullptr, nullptr, 0, status, st),
           "center");
    }
    if (tm) CK(cudaEventRecord(ws->ev[3], st), "event");
    Arena sa{static_cast<char*>(w.solve), w.solve_bytes, 0};
    // narrow blocks: parameter-space Gram on compact rows, solve on compact offsets
    if (wp.nnar > 0) {
        GramTable* tab = new (std::nothrow) GramTable;
        if (!tab) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
        tab->nb = wp.nnar;
        tab->total_tiles = 0;
        long long so = 0;
        for (int i = 0; i < wp.nnar; ++i) {
            const int b = wp.nar[i];
            const long long n = off[b + 1] - off[b], T = (n + 63) / 64;
            GBlk& g = tab->b[i];
            g.row0 = nsp ? wp.nar_off[i] : off[b];
            g.s_off = so;
            g.n = (int)n;
            g.tiles = (int)(T * (T + 1) / 2);
            g.tile0 = tab->total_tiles;
            g.scale = 0.0;
            tab->total_tiles += T * (T + 1) / 2;
            so += n * n;
        }
        cudaError_t e;
        if (nsp) {
            e = launch_gram_tc(nsp, w.planes, w.gexp, wp.nar_np, 2 * wp.nar_np, w.ldk, w.ldk, 1.0 / (double)ns, *tab,
                               w.S, status, st);
            if (e == cudaSuccess) e = launch_set_diag(w.S, *tab, w.diag, st);
        } else {
            e = launch_gram_simt(prec, w.O, w.ldo, ns, nullptr, 1.0 / (double)ns, *tab, w.S, st);
        }
        delete tab;
        if (e == cudaErrorNotSupported) return fail(NQS_ERR_UNSUPPORTED, "tensor-core Gram needs an sm_103 device");
        CK(e, "gram");
        for (int i = 0; i < wp.nnar; ++i) {
            const int b = wp.nar[i];
            CK(cudaMemcpyAsync(w.Fn + wp.nar_off[i], w.F + off[b], 16 * (size_t)(off[b + 1] - off[b]),
                               cudaMemcpyDeviceToDevice, st),
               "gather F");
        }
        int32_t* nk = n_kept ? w.nkn : nullptr;
        Arena sa2 = sa;
        rc = run_solve(w.S, wp.nar_off, wp.nnar, w.Fn, shift, cutoff, mode, eta,
                       solver == NQS_SOLVE_MIXED ? NQS_SOLVE_MIXED_PSD : solver, w.dthn, nullptr, nk, sa2, status, st,
                       nullptr, nullptr, graph, step_ref_tol(prec));
        if (rc) return rc;
        for (int i = 0; i < wp.nnar; ++i) {
            const int b = wp.nar[i];
            CK(cudaMemcpyAsync(dtheta + off[b], w.dthn + wp.nar_off[i], 16 * (size_t)(off[b + 1] - off[b]),
                               cudaMemcpyDeviceToDevice, st),
               "scatter dtheta");
            if (nk) CK(cudaMemcpyAsync(n_kept + b, nk + i, 4, cudaMemcpyDeviceToDevice, st), "n_kept");
        }
    }
    // wide blocks, one at a time: sample-space Gram, solve, back-projection
    const int64_t offT[2] = {0, ns};
    for (int i = 0; i < wp.nwide; ++i) {
        const int b = wp.wid[i];
        const long long n = off[b + 1] - off[b];
        const c128* dOb = reinterpret_cast<const c128*>(Ob + cs * (size_t)off[b] * (size_t)w.ldo);
        GramTable* tab = new (std::nothrow) GramTable;
        if (!tab) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
        gram_table(offT, 1, 64, tab);
        cudaError_t e;
        if (nsp) {
            e = launch_transpose_group(dOb, w.ldo, ns, n, w.planesT, w.gexpT, w.ldkT, w.diagT, st);
            if (e == cudaSuccess)
                e = launch_gram_tc(nsp, w.planesT, w.gexpT, ns, 2 * ns, w.ldkT, w.ldkT, 1.0 / (double)ns, *tab, w.T,
                                   status, st);
            if (e == cudaSuccess) e = launch_set_diag(w.T, *tab, w.diagT, st);
        } else {
            e = launch_ntk_transpose(NQS_FP64, dOb, w.ldo, ns, n, w.Y, w.ldy, st);
            if (e == cudaSuccess) e = launch_gram_simt(NQS_FP64, w.Y, w.ldy, w.ldy, nullptr, 1.0 / (double)ns, *tab,
                                                       w.T, st);
        }
        delete tab;
        if (e == cudaErrorNotSupported) return fail(NQS_ERR_UNSUPPORTED, "tensor-core Gram needs an sm_103 device");
        CK(e, "sample-space gram");
        // the Gram kernels give conj(X X^H): solve (conj(X X^H) + lambda I) u = conj(eps), then
        // dtheta_b = -eta X^H conj(u)
        CK(launch_ntk_rhs(w.e, ns, w.rhs, st), "rhs");
        Arena sa2 = sa;
        rc = run_solve(w.T, offT, 1, w.rhs, shift, cutoff, mode, -1.0, NQS_SOLVE_MIXED_PSD, w.u, nullptr, w.keptT, sa2,
                       status, st, nullptr, nullptr, graph, step_ref_tol(prec));
        if (rc) return rc;
        CK(launch_ntk_back(dOb, w.ldo, ns, n, w.u, eta, dtheta + off[b], st), "back-projection");
        if (n_kept) {
            count_launch();
            wide_kept_kernel<<<1, 32, 0, st>>>(w.keptT, ns, n, n_kept + b);
            CK(cudaGetLastError(), "n_kept");
        }
    }
    if (tm) {
        CK(cudaEventRecord(ws->ev[4], st), "event");
        CK(cudaEventRecord(ws->ev[5], st), "event");
        CK(cudaEventRecord(ws->ev[6], st), "event");
        ws->recorded = true;
    }
    return NQS_OK;
}

}  // namespace

extern "C" {

const char* nqs_last_error(void) { return g_err.c_str(); }
const char* nqs_version(void) { return "nqs_sr 0.1 (sm_103a)"; }

int nqs_workspace_create(void* device_ptr, size_t bytes, nqs_workspace** ws) {
    if (!ws || !device_ptr) return fail(NQS_ERR_INVALID_ARG, "NULL workspace pointer");
    if (reinterpret_cast<uintptr_t>(device_ptr) % 256) return fail(NQS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (bytes < STATUS_BYTES) return fail(NQS_ERR_WORKSPACE, "workspace smaller than %zu bytes", STATUS_BYTES);
    nqs_workspace* w = new (std::nothrow) nqs_workspace;
    if (!w) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
    w->base = static_cast<char*>(device_ptr);
    w->bytes = bytes;
    w->timing = false;
    w->recorded = false;
    for (int i = 0; i <= NSTAGE; ++i) w->ev[i] = nullptr;
    cudaError_t e = cudaMemset(w->base, 0, STATUS_BYTES);
    if (e != cudaSuccess) {
        delete w;
        return cuda_fail(e, "workspace status init");
    }
    *ws = w;
    return NQS_OK;
}

int nqs_workspace_destroy(nqs_workspace* ws) {
    if (ws) {
        for (int i = 0; i <= NSTAGE; ++i)
            if (ws->ev[i]) cudaEventDestroy(ws->ev[i]);
    }
    delete ws;
    return NQS_OK;
}

int nqs_stage_timing(nqs_workspace* ws, int32_t enable) {
    if (!ws) return fail(NQS_ERR_INVALID_ARG, "workspace is NULL");
    if (enable && !ws->ev[0]) {
        for (int i = 0; i <= NSTAGE; ++i) CK(cudaEventCreate(&ws->ev[i]), "event create");
    }
    ws->timing = enable != 0;
    ws->recorded = false;
    return NQS_OK;
}

int nqs_stage_times(nqs_workspace* ws, double* ms_out, int32_t max_stages, int32_t* n_stages) {
    if (!ws || !ms_out || !n_stages) return fail(NQS_ERR_INVALID_ARG, "NULL argument");
    if (!ws->recorded) return fail(NQS_ERR_INVALID_ARG, "no timed sr_step since timing was enabled");
    CK(cudaEventSynchronize(ws->ev[NSTAGE]), "event sync");
    const int n = max_stages < NSTAGE ? max_stages : NSTAGE;
    for (int i = 0; i < n; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ws->ev[i], ws->ev[i + 1]), "elapsed");
        ms_out[i] = ms;
    }
    *n_stages = n;
    return NQS_OK;
}

int nqs_set_gram_tuning(int32_t n, const int64_t* max_nb, const int64_t* max_ns, const int32_t* group) {
    if (n < 0 || n > GRAM_TUNE_MAX || (n > 0 && (!max_nb || !max_ns || !group)))
        return fail(NQS_ERR_INVALID_ARG, "nqs_set_gram_tuning: 0 <= n <= %d entries with non-NULL arrays",
                    GRAM_TUNE_MAX);
    for (int i = 0; i < n; ++i)
        if (group[i] < 1 || group[i] > 64 || max_nb[i] < 1 || max_ns[i] < 1)
            return fail(NQS_ERR_INVALID_ARG, "nqs_set_gram_tuning: entry %d out of range", i);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_n = n;
    for (int i = 0; i < n; ++i) g_tune[i] = GramTune{max_nb[i], max_ns[i], group[i]};
    return NQS_OK;
}

int32_t nqs_gram_group_edge(int64_t max_nb, int64_t n_s) { return gram_group_edge(max_nb, n_s); }

int nqs_set_limits(int32_t max_sweeps, int64_t wait_ns) {
    if (max_sweeps < 0 || wait_ns < 0) return fail(NQS_ERR_INVALID_ARG, "nqs_set_limits: negative limit");
    g_ql_maxit.store(max_sweeps ? max_sweeps : QL_MAXIT_DEFAULT);
    g_ref_maxit.store(max_sweeps ? max_sweeps : REF_MAXIT_DEFAULT);
    g_wait_ns.store(wait_ns ? (unsigned long long)wait_ns : WAIT_NS_DEFAULT);
    return NQS_OK;
}

int nqs_set_eloc_fallback_all(int32_t on) {
    g_dp_fallback_all.store(on ? 1 : 0);
    return NQS_OK;
}

int64_t nqs_launch_count(void) { return (int64_t)__atomic_load_n(&launch_counter(), __ATOMIC_RELAXED); }

int nqs_sync_status(nqs_workspace* ws, void* stream) {
    if (!ws) return fail(NQS_ERR_INVALID_ARG, "workspace is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus h;
    CK(cudaMemcpyAsync(&h, ws->base, sizeof h, cudaMemcpyDeviceToHost, st), "status read");
    CK(cudaStreamSynchronize(st), "stream sync");
    if (h.code != 0) {
        CK(cudaMemsetAsync(ws->base, 0, sizeof(DevStatus), st), "status clear");
        CK(cudaStreamSynchronize(st), "stream sync");
        return fail(h.code, "device reported status %d in stage %d (detail %lld)", h.code, h.where, h.detail);
    }
    return NQS_OK;
}

int64_t qgt_packed_size(const int64_t* block_off, int32_t n_blocks) {
    if (!block_off || n_blocks < 1) return -1;
    int64_t t = 0;
    for (int b = 0; b < n_blocks; ++b) t += (block_off[b + 1] - block_off[b]) * (block_off[b + 1] - block_off[b]);
    return t;
}

// ---------------------------------------------------------------- sizes
int nqs_jacobian_workspace_size(const nqs_model* m, int64_t n_s, int32_t precision, size_t* bytes) {
    ModelDesc md;
    if (!bytes || n_s < 1 || check_prec(precision)) return fail(NQS_ERR_INVALID_ARG, "bad arguments");
    if (build_model_desc(m, n_s, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (md.kind == NQS_VIT && precision == NQS_FP32)
        return fail(NQS_ERR_UNSUPPORTED, "the transformer runs in FP64 only (not NQS_FP32)");
    Arena a = sizing_arena();
    JacBufs jb;
    plan_model(a, md, n_s, jac_prec(precision), &jb, true);
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

int nqs_local_energy_workspace_size(const nqs_model* m, int64_t n_s, const nqs_hamiltonian* h, int32_t precision,
                                    size_t* bytes) {
    ModelDesc md;
    if (!bytes || n_s < 1 || !h || check_prec(precision)) return fail(NQS_ERR_INVALID_ARG, "bad arguments");
    if (build_model_desc(m, n_s, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (md.kind == NQS_VIT && precision == NQS_FP32)
        return fail(NQS_ERR_UNSUPPORTED, "the transformer runs in FP64 only (not NQS_FP32)");
    Arena a = sizing_arena();
    JacBufs jb;
    plan_model(a, md, n_s, eloc_prec(precision), &jb, false);
    ElocBufs eb;
    plan_eloc(a, md, n_s, h->n_bonds, &eb);
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

int qgt_block_build_workspace_size(int64_t n_s, int64_t n_p, const int64_t* block_off, int32_t n_blocks,
                                   int32_t precision, size_t* bytes) {
    if (!bytes || n_s < 1 || check_prec(precision)) return fail(NQS_ERR_INVALID_ARG, "bad arguments");
    int rc = check_offsets(block_off, n_blocks, n_p);
    if (rc) return rc;
    Arena a = sizing_arena();
    BuildBufs bb;
    plan_build(a, n_s, n_p, precision, &bb);
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

int qgt_block_solve_workspace_size(const int64_t* block_off, int32_t n_blocks, size_t* bytes) {
    if (!bytes) return fail(NQS_ERR_INVALID_ARG, "bytes is NULL");
    int rc = check_offsets(block_off, n_blocks, -1);
    if (rc) return rc;
    *bytes = al256(solve_workspace_bytes(block_off, n_blocks)) + STATUS_BYTES;
    return NQS_OK;
}

static void plan_step(Arena& a, const ModelDesc& md, long long ns, int nbonds, const int64_t* off, int nb, int prec,
                      JacBufs* jb, JacBufs* jbe, ElocBufs* eb, BuildBufs* bb, void** O, long long* ldo, c128** eloc,
                      c128** F, c128** S) {
    plan_model(a, md, ns, jac_prec(prec), jb, true);
    if (eloc_prec(prec) != jac_prec(prec)) plan_model(a, md, ns, eloc_prec(prec), jbe, false);
    else *jbe = *jb;
    plan_eloc(a, md, ns, nbonds, eb);
    plan_build(a, ns, md.n_p, prec, bb);
    *ldo = round_up(ns, 32);
    *O = a.take(csize(prec) * (size_t)md.n_p * (size_t)(*ldo));
    *eloc = static_cast<c128*>(a.take(16 * ns));
    *F = static_cast<c128*>(a.take(16 * (size_t)md.n_p));
    long long sz = 0;
    for (int b = 0; b < nb; ++b) sz += (off[b + 1] - off[b]) * (off[b + 1] - off[b]);
    *S = static_cast<c128*>(a.take(16 * (size_t)sz));
}

int sr_step_workspace_size(const nqs_model* m, int64_t n_s, const nqs_hamiltonian* h, const int64_t* block_off,
                           int32_t n_blocks, int32_t precision, size_t* bytes) {
    ModelDesc md;
    if (!bytes || n_s < 1 || !h || check_prec(precision)) return fail(NQS_ERR_INVALID_ARG, "bad arguments");
    if (build_model_desc(m, n_s, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (md.kind == NQS_VIT && precision == NQS_FP32)
        return fail(NQS_ERR_UNSUPPORTED, "the transformer runs in FP64 only (not NQS_FP32)");
    int rc = check_offsets(block_off, n_blocks, md.n_p);
    if (rc) return rc;
    Arena a = sizing_arena();
    JacBufs jb, jbe;
    ElocBufs eb;
    BuildBufs bb;
    void* O;
    long long ldo;
    c128 *eloc, *F, *S;
    plan_step(a, md, n_s, h->n_bonds, block_off, n_blocks, precision, &jb, &jbe, &eb, &bb, &O, &ldo, &eloc, &F, &S);
    a.take(solve_workspace_bytes(block_off, n_blocks));
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

int sr_step_workspace_size2(const nqs_model* m, int64_t n_s, const nqs_hamiltonian* h, const int64_t* block_off,
                            int32_t n_blocks, double diag_shift, int32_t precision, int32_t solver, int32_t flags,
                            size_t* bytes) {
    ModelDesc md;
    if (!bytes || n_s < 1 || !h || check_prec(precision)) return fail(NQS_ERR_INVALID_ARG, "bad arguments");
    if (build_model_desc(m, n_s, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (md.kind == NQS_VIT && precision == NQS_FP32)
        return fail(NQS_ERR_UNSUPPORTED, "the transformer runs in FP64 only (not NQS_FP32)");
    int rc = check_offsets(block_off, n_blocks, md.n_p);
    if (rc) return rc;
    WidePlan* wp = new (std::nothrow) WidePlan;
    if (!wp) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
    wide_plan(block_off, n_blocks, n_s, diag_shift, precision, solver, flags, wp);
    if (wp->nwide == 0) {
        delete wp;
        return sr_step_workspace_size(m, n_s, h, block_off, n_blocks, precision, bytes);
    }
    Arena a = sizing_arena();
    WideBufs wb;
    plan_wide(a, md, n_s, h->n_bonds, block_off, n_blocks, precision, *wp, &wb);
    delete wp;
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

// ---------------------------------------------------------------- compute calls
int nqs_jacobian(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s, int32_t precision,
                 void* logpsi_out, void* O_out, int64_t ldo, nqs_workspace* ws, void* stream) {
    ModelDesc md;
    if (check_prec(precision)) return NQS_ERR_INVALID_ARG;
    if (n_s < 1 || !theta || !configs || !logpsi_out || !O_out || ldo < n_s)
        return fail(NQS_ERR_INVALID_ARG, "nqs_jacobian: NULL pointer, n_s < 1 or ldo < n_s");
    if (build_model_desc(m, n_s, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (md.kind == NQS_VIT && precision == NQS_FP32)
        return fail(NQS_ERR_UNSUPPORTED, "the transformer runs in FP64 only (not NQS_FP32)");
    Arena a = arena_of(ws);
    JacBufs jb;
    plan_model(a, md, n_s, jac_prec(precision), &jb, true);
    int rc = check_ws(ws, a);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rp = jac_prec(precision);
    rc = run_model(md, rp, theta, configs, n_s, jb, st);
    if (rc) return rc;
    CK(launch_backward(rp, md, jb.thR, jb.Z, n_s, jb.G, st), "backward");
    CK(launch_jac_write(rp, md, jb.thR, jb.Z, jb.G, configs, n_s, O_out, ldo, st), "jacobian");
    CK(cudaMemcpyAsync(logpsi_out, jb.logpsi, sizeof(c128) * n_s, cudaMemcpyDeviceToDevice, st), "logpsi copy");
    return NQS_OK;
}

int nqs_vjp(const void* O, int64_t ldo, int64_t n_s, int64_t n_p, int32_t precision, const void* g, void* out,
            void* stream) {
    if (check_prec(precision)) return NQS_ERR_INVALID_ARG;
    if (!O || !g || !out || n_s < 1 || n_p < 1 || ldo < n_s) return fail(NQS_ERR_INVALID_ARG, "nqs_vjp: bad arguments");
    CK(launch_vjp(jac_prec(precision), O, ldo, n_s, n_p, static_cast<const c128*>(g), static_cast<c128*>(out),
                  static_cast<cudaStream_t>(stream)),
       "vjp");
    return NQS_OK;
}

int nqs_local_energy(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s,
                     const nqs_hamiltonian* h, int32_t precision, void* eloc_out, nqs_workspace* ws, void* stream) {
    return nqs_local_energy_ex(m, theta, configs, n_s, h, precision, 0, eloc_out, ws, stream);
}

int nqs_local_energy_ex(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s,
                        const nqs_hamiltonian* h, int32_t precision, int32_t flags, void* eloc_out,
                        nqs_workspace* ws, void* stream) {
    ModelDesc md;
    HamDesc hd;
    if (check_prec(precision)) return NQS_ERR_INVALID_ARG;
    if ((flags & ~NQS_ELOC_DIFF32) || ((flags & NQS_ELOC_DIFF32) && precision == NQS_FP32))
        return fail(NQS_ERR_INVALID_ARG, "nqs_local_energy_ex: bad flags (NQS_ELOC_DIFF32 needs an FP64 forward)");
    if (n_s < 1 || !theta || !configs || !eloc_out) return fail(NQS_ERR_INVALID_ARG, "nqs_local_energy: bad arguments");
    if (build_model_desc(m, n_s, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (md.kind == NQS_VIT && precision == NQS_FP32)
        return fail(NQS_ERR_UNSUPPORTED, "the transformer runs in FP64 only (not NQS_FP32)");
    int rc = ham_desc(h, md.N, &hd);
    if (rc) return rc;
    Arena a = arena_of(ws);
    JacBufs jb;
    const int rp = eloc_prec(precision);
    plan_model(a, md, n_s, rp, &jb, false);
    ElocBufs eb;
    plan_eloc(a, md, n_s, hd.n_bonds, &eb);
    rc = check_ws(ws, a);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = run_model(md, rp, theta, configs, n_s, jb, st);
    if (rc) return rc;
    return run_eloc(md, rp, hd, configs, n_s, jb, eb, static_cast<c128*>(eloc_out), status_of(ws), st,
                    eloc_dp(precision, flags));
}

int nqs_metropolis_workspace_size(const nqs_model* m, int64_t n_chains, size_t* bytes) {
    ModelDesc md;
    if (!bytes || n_chains < 1) return fail(NQS_ERR_INVALID_ARG, "nqs_metropolis_workspace_size: bad arguments");
    if (build_model_desc(m, n_chains, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    Arena a = sizing_arena();
    McBufs b;
    plan_mc(a, md, n_chains, &b);
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

int nqs_metropolis(const nqs_model* m, const void* theta, int8_t* configs, int64_t n_chains, int32_t n_steps,
                   const double* uniforms, int64_t* n_accepted, nqs_workspace* ws, void* stream) {
    ModelDesc md;
    if (n_chains < 1 || n_steps < 0 || !theta || !configs || (n_steps > 0 && !uniforms))
        return fail(NQS_ERR_INVALID_ARG, "nqs_metropolis: bad arguments");
    if (build_model_desc(m, n_chains, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (n_chains > 2147483647LL) return fail(NQS_ERR_INVALID_ARG, "nqs_metropolis: more than 2^31 - 1 chains");
    Arena a = arena_of(ws);
    McBufs b;
    plan_mc(a, md, n_chains, &b);
    int rc = check_ws(ws, a);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(n_accepted);
    if (acc) CK(cudaMemsetAsync(acc, 0, sizeof(*acc), st), "memset");
    if (n_steps == 0) return NQS_OK;
    CK(launch_prepare_params(NQS_FP64, md, theta, b.jb.thR, b.jb.wtR, st), "prepare_params");
    CK(launch_split_weights(md, b.jb.wtR, b.wdf, st), "split_weights");
    CK(launch_mc_setup(n_chains, b.bond_J, b.csamp, b.cbond, b.nconn, st), "mc_setup");
    HamDesc hd;
    hd.n_sites = md.N;
    hd.n_bonds = (int)n_chains;
    hd.bond_ij = b.pairs;
    hd.bond_J = b.bond_J;
    hd.c = 1.0;
    hd.sign_rule = 1;
    for (int t = 0; t < n_steps; ++t) {
        const double* u = uniforms + (size_t)3 * (size_t)n_chains * (size_t)t;
        CK(launch_forward(NQS_FP64, md, b.jb.thR, b.jb.wtR, configs, n_chains, b.jb.Z, b.jb.logpsi, st), "forward");
        CK(launch_mc_propose(configs, md.N, n_chains, u, b.pairs, b.valid, st), "mc_propose");
        CK(launch_conn_terms(NQS_FP64, md, b.jb.thR, b.jb.wtR, b.wdf, b.jb.Z, b.jb.logpsi, configs, hd, b.cbond,
                             b.csamp, b.nconn, n_chains, b.ratio, st),
           "ratios");
        CK(launch_mc_accept(configs, md.N, n_chains, u, b.pairs, b.valid, b.ratio, acc, st), "mc_accept");
    }
    return NQS_OK;
}

int nqs_theta_update(void* theta, const void* dtheta, int64_t n_p, void* stream) {
    if (!theta || !dtheta || n_p < 0) return fail(NQS_ERR_INVALID_ARG, "nqs_theta_update: bad arguments");
    CK(launch_theta_update(static_cast<c128*>(theta), static_cast<const c128*>(dtheta), n_p,
                           static_cast<cudaStream_t>(stream)),
       "theta_update");
    return NQS_OK;
}

int nqs_connections(const int8_t* configs, int64_t n_s, const nqs_hamiltonian* h, int32_t* conn_count,
                    int64_t* conn_offset, int32_t* conn_bond, int64_t max_conn, int64_t* n_conn_out,
                    nqs_workspace* ws, void* stream) {
    HamDesc hd;
    if (!configs || n_s < 1 || !conn_count || !conn_offset || !conn_bond || !n_conn_out)
        return fail(NQS_ERR_INVALID_ARG, "nqs_connections: bad arguments");
    if (!h) return fail(NQS_ERR_INVALID_ARG, "hamiltonian is NULL");
    int rc = ham_desc(h, h->n_sites, &hd);
    if (rc) return rc;
    if (hd.n_sites < 2 || hd.n_sites > MAXN) return fail(NQS_ERR_INVALID_ARG, "bad n_sites");
    Arena a = arena_of(ws);
    int32_t* csamp = static_cast<int32_t*>(a.take(4 * (size_t)(max_conn > 0 ? max_conn : 1)));
    rc = check_ws(ws, a);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(launch_conn_count(configs, n_s, hd, conn_count, status_of(ws), st), "conn_count");
    CK(launch_scan(conn_count, n_s, reinterpret_cast<long long*>(conn_offset), st), "scan");
    long long total = 0;
    CK(cudaMemcpyAsync(&total, conn_offset + n_s, sizeof total, cudaMemcpyDeviceToHost, st), "total read");
    CK(cudaStreamSynchronize(st), "sync");
    *n_conn_out = total;
    if (total > max_conn) return fail(NQS_ERR_INVALID_ARG, "max_conn %lld < %lld connections", (long long)max_conn, total);
    CK(launch_conn_fill(configs, n_s, hd, reinterpret_cast<const long long*>(conn_offset), conn_bond, csamp, st),
       "conn_fill");
    return NQS_OK;
}

int qgt_block_build(void* O, int64_t ldo, int64_t n_s, int64_t n_p, const double* w, const int64_t* block_off,
                    int32_t n_blocks, const void* eloc, int32_t precision, void* S_packed, void* F_out,
                    void* Omean_out, void* Emean_out, nqs_workspace* ws, void* stream) {
    if (check_prec(precision)) return NQS_ERR_INVALID_ARG;
    if (!O || !eloc || !S_packed || !F_out || n_s < 1 || n_p < 1 || ldo < n_s)
        return fail(NQS_ERR_INVALID_ARG, "qgt_block_build: bad arguments");
    int rc = check_offsets(block_off, n_blocks, n_p);
    if (rc) return rc;
    Arena a = arena_of(ws);
    BuildBufs bb;
    plan_build(a, n_s, n_p, precision, &bb);
    rc = check_ws(ws, a);
    if (rc) return rc;
    return run_build(O, ldo, n_s, n_p, w, block_off, n_blocks, static_cast<const c128*>(eloc), precision,
                     static_cast<c128*>(S_packed), static_cast<c128*>(F_out), static_cast<c128*>(Omean_out),
                     static_cast<c128*>(Emean_out), bb, status_of(ws), static_cast<cudaStream_t>(stream));
}

int nqs_shard_sums(const void* O, int64_t ldo, int64_t n_s, int64_t n_p, int32_t precision, const void* eloc,
                   void* osum_out, void* esum_out, void* stream) {
    if (check_prec(precision)) return NQS_ERR_INVALID_ARG;
    if (!O || !eloc || !osum_out || !esum_out || n_s < 1 || n_p < 1 || ldo < n_s)
        return fail(NQS_ERR_INVALID_ARG, "nqs_shard_sums: bad arguments");
    CK(launch_shard_sums(jac_prec(precision), O, ldo, n_s, n_p, static_cast<const c128*>(eloc),
                         static_cast<c128*>(osum_out), static_cast<c128*>(esum_out), static_cast<cudaStream_t>(stream)),
       "shard sums");
    return NQS_OK;
}

int qgt_block_build_shard(void* O, int64_t ldo, int64_t n_s, int64_t n_p, int64_t n_total, const int64_t* block_off,
                          int32_t n_blocks, const void* eloc, const void* Osum_in, const void* Esum_in,
                          int32_t precision, void* S_packed, void* F_out, void* Omean_out, void* Emean_out,
                          nqs_workspace* ws, void* stream) {
    if (check_prec(precision)) return NQS_ERR_INVALID_ARG;
    if (!O || !eloc || !Osum_in || !Esum_in || !S_packed || !F_out || n_s < 1 || n_p < 1 || ldo < n_s ||
        n_total < n_s)
        return fail(NQS_ERR_INVALID_ARG, "qgt_block_build_shard: bad arguments");
    const double weight = 1.0 / (double)n_total;
    int rc = check_offsets(block_off, n_blocks, n_p);
    if (rc) return rc;
    Arena a = arena_of(ws);
    BuildBufs bb;
    plan_build(a, n_s, n_p, precision, &bb);
    rc = check_ws(ws, a);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus* status = status_of(ws);
    const int nsp = nsplit_of(precision);
    c128* S = static_cast<c128*>(S_packed);
    CK(launch_sums_to_means(static_cast<const c128*>(Osum_in), static_cast<const c128*>(Esum_in), n_p, n_total,
                            bb.means, st),
       "means");
    if (Omean_out)
        CK(cudaMemcpyAsync(Omean_out, bb.means, 16 * (size_t)n_p, cudaMemcpyDeviceToDevice, st), "mean copy");
    if (Emean_out)
        CK(cudaMemcpyAsync(Emean_out, bb.means + n_p, 16, cudaMemcpyDeviceToDevice, st), "mean copy");
    CK(launch_ecenter(static_cast<const c128*>(eloc), n_s, bb.means + n_p, bb.e, st), "ecenter");
    CK(launch_center(precision, nsp, O, ldo, n_s, n_p, nullptr, bb.e, static_cast<c128*>(F_out), nullptr,
                     nsp ? bb.planes : nullptr, bb.ldk, bb.diag, bb.gexp, n_p, status, st, bb.means, weight),
       "center");
    GramTable* tab = new (std::nothrow) GramTable;
    if (!tab) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
    gram_table(block_off, n_blocks, 64, tab);
    cudaError_t e;
    if (nsp) {
        e = launch_gram_tc(nsp, bb.planes, bb.gexp, n_p, 2 * n_p, bb.ldk, bb.ldk, weight, *tab, S, status, st);
        if (e == cudaSuccess) e = launch_set_diag(S, *tab, bb.diag, st);
    } else {
        e = launch_gram_simt(precision, O, ldo, n_s, nullptr, weight, *tab, S, st);
    }
    delete tab;
    if (e == cudaErrorNotSupported) return fail(NQS_ERR_UNSUPPORTED, "tensor-core Gram needs an sm_103 device");
    CK(e, "gram");
    return NQS_OK;
}

static void plan_ntk(Arena& a, long long ns, long long np, int prec, c128** e, c128** F, void** Y, long long* ldy,
                     c128** S, c128** rhs, c128** u) {
    *e = static_cast<c128*>(a.take(16 * (size_t)ns));
    *F = static_cast<c128*>(a.take(16 * (size_t)np));
    *ldy = round_up(np, 32);
    *Y = a.take(csize(prec) * (size_t)ns * (size_t)(*ldy));
    *S = static_cast<c128*>(a.take(16 * (size_t)ns * (size_t)ns));
    *rhs = static_cast<c128*>(a.take(16 * (size_t)ns));
    *u = static_cast<c128*>(a.take(16 * (size_t)ns));
}

int ntk_solve_workspace_size(int64_t n_s, int64_t n_p, int32_t precision, size_t* bytes) {
    if (!bytes || n_s < 1 || n_p < 1 || (precision != NQS_FP64 && precision != NQS_FP32))
        return fail(NQS_ERR_INVALID_ARG, "ntk_solve_workspace_size: bad arguments");
    Arena a = sizing_arena();
    c128 *e, *F, *S, *rhs, *u;
    void* Y;
    long long ldy;
    plan_ntk(a, n_s, n_p, precision, &e, &F, &Y, &ldy, &S, &rhs, &u);
    const int64_t off[2] = {0, n_s};
    a.take(solve_workspace_bytes(off, 1));
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

int ntk_solve(void* O, int64_t ldo, int64_t n_s, int64_t n_p, const void* eloc, double diag_shift, double cutoff,
              double eta, int32_t precision, void* dtheta_out, void* Emean_out, nqs_workspace* ws, void* stream) {
    if (precision != NQS_FP64 && precision != NQS_FP32)
        return fail(NQS_ERR_INVALID_ARG, "ntk_solve: precision must be NQS_FP64 or NQS_FP32");
    if (!O || !eloc || !dtheta_out || n_s < 1 || n_p < 1 || ldo < n_s)
        return fail(NQS_ERR_INVALID_ARG, "ntk_solve: bad arguments");
    Arena a = arena_of(ws);
    c128 *e, *F, *S, *rhs, *u;
    void* Y;
    long long ldy;
    plan_ntk(a, n_s, n_p, precision, &e, &F, &Y, &ldy, &S, &rhs, &u);
    const int64_t off[2] = {0, n_s};
    Arena need = a;
    need.take(solve_workspace_bytes(off, 1));
    int rc = check_ws(ws, need);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus* status = status_of(ws);
    CK(launch_emean(static_cast<const c128*>(eloc), nullptr, n_s, static_cast<c128*>(Emean_out), e, status, st),
       "emean");
    CK(launch_center(NQS_FP64, 0, O, ldo, n_s, n_p, nullptr, e, F, nullptr, nullptr, 0, nullptr, nullptr, n_p, status,
                     st),
       "center");
    CK(launch_ntk_transpose(precision, static_cast<const c128*>(O), ldo, n_s, n_p, Y, ldy, st), "transpose");
    GramTable* tab = new (std::nothrow) GramTable;
    if (!tab) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
    gram_table(off, 1, 64, tab);
    cudaError_t err = launch_gram_simt(precision, Y, ldy, ldy, nullptr, 1.0 / (double)n_s, *tab, S, st);
    delete tab;
    CK(err, "sample gram");
    CK(launch_ntk_rhs(e, n_s, rhs, st), "rhs");
    // u = (S_T + lambda I)^{-1} conj(eps): the block solver's dtheta with eta = -1
    rc = run_solve(S, off, 1, rhs, diag_shift, cutoff, 0, -1.0,
                   precision == NQS_FP64 ? NQS_SOLVE_FP64 : NQS_SOLVE_MIXED_PSD, u, nullptr, nullptr, a, status, st);
    if (rc) return rc;
    CK(launch_ntk_back(static_cast<const c128*>(O), ldo, n_s, n_p, u, eta, static_cast<c128*>(dtheta_out), st),
       "back");
    return NQS_OK;
}

int qgt_block_solve(void* S_packed, const int64_t* block_off, int32_t n_blocks, const void* F, double diag_shift,
                    double cutoff, int32_t cutoff_mode, double eta, int32_t solver, void* dtheta_out,
                    double* evals_out, int32_t* n_kept_out, nqs_workspace* ws, void* stream) {
    if (!S_packed || !F || !dtheta_out) return fail(NQS_ERR_INVALID_ARG, "qgt_block_solve: NULL pointer");
    int rc = check_offsets(block_off, n_blocks, -1);
    if (rc) return rc;
    Arena a = arena_of(ws);
    Arena need = sizing_arena();
    need.take(solve_workspace_bytes(block_off, n_blocks));
    rc = check_ws(ws, need);
    if (rc) return rc;
    return run_solve(static_cast<c128*>(S_packed), block_off, n_blocks, static_cast<const c128*>(F), diag_shift,
                     cutoff, cutoff_mode, eta, solver, static_cast<c128*>(dtheta_out), evals_out, n_kept_out, a,
                     status_of(ws), static_cast<cudaStream_t>(stream));
}

int sr_step(const nqs_model* m, const void* theta, const int8_t* configs, int64_t n_s, const nqs_hamiltonian* h,
            const int64_t* block_off, int32_t n_blocks, double diag_shift, double cutoff, int32_t cutoff_mode,
            double eta, int32_t precision, int32_t solver, void* dtheta_out, void* Emean_out, double* evals_out,
            int32_t* n_kept_out, int32_t flags, nqs_workspace* ws, void* stream) {
    ModelDesc md;
    HamDesc hd;
    if (check_prec(precision)) return NQS_ERR_INVALID_ARG;
    if (n_s < 1 || !theta || !configs || !dtheta_out || !Emean_out)
        return fail(NQS_ERR_INVALID_ARG, "sr_step: bad arguments");
    if ((flags & NQS_ELOC_DIFF32) && precision == NQS_FP32)
        return fail(NQS_ERR_INVALID_ARG, "sr_step: NQS_ELOC_DIFF32 needs an FP64 forward (not NQS_FP32)");
    if (build_model_desc(m, n_s, &md)) return fail(NQS_ERR_INVALID_ARG, "bad model description");
    if (md.kind == NQS_VIT && precision == NQS_FP32)
        return fail(NQS_ERR_UNSUPPORTED, "the transformer runs in FP64 only (not NQS_FP32)");
    int rc = ham_desc(h, md.N, &hd);
    if (rc) return rc;
    rc = check_offsets(block_off, n_blocks, md.n_p);
    if (rc) return rc;
    const bool graph = (flags & NQS_GRAPH) != 0;
    if (graph && (flags & NQS_SYNC)) return fail(NQS_ERR_INVALID_ARG, "NQS_GRAPH cannot be combined with NQS_SYNC");
    {
        WidePlan* wp = new (std::nothrow) WidePlan;
        if (!wp) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
        wide_plan(block_off, n_blocks, n_s, diag_shift, precision, solver, flags, wp);
        if (wp->nwide > 0) {
            if (solver != NQS_SOLVE_MIXED && solver != NQS_SOLVE_MIXED_PSD) {
                delete wp;
                return fail(NQS_ERR_INVALID_ARG, "unknown solver %d", solver);
            }
            if (evals_out) {
                delete wp;
                return fail(NQS_ERR_UNSUPPORTED, "eigenvalues of a block wider than N_s: call with NQS_PARAM_SPACE");
            }
            Arena a = arena_of(ws);
            WideBufs wb;
            plan_wide(a, md, n_s, hd.n_bonds, block_off, n_blocks, precision, *wp, &wb);
            rc = check_ws(ws, a);
            if (!rc)
                rc = run_step_wide(md, hd, theta, configs, n_s, block_off, n_blocks, diag_shift, cutoff, cutoff_mode,
                                   eta, precision, solver, static_cast<c128*>(dtheta_out), static_cast<c128*>(Emean_out),
                                   n_kept_out, flags, *wp, wb, ws, status_of(ws), static_cast<cudaStream_t>(stream));
            delete wp;
            if (rc) return rc;
            if (flags & NQS_SYNC) return nqs_sync_status(ws, stream);
            return NQS_OK;
        }
        delete wp;
    }
    Arena a = arena_of(ws);
    JacBufs jb, jbe;
    ElocBufs eb;
    BuildBufs bb;
    void* O;
    long long ldo;
    c128 *eloc, *F, *S;
    plan_step(a, md, n_s, hd.n_bonds, block_off, n_blocks, precision, &jb, &jbe, &eb, &bb, &O, &ldo, &eloc, &F, &S);
    Arena need = a;
    need.take(solve_workspace_bytes(block_off, n_blocks));
    rc = check_ws(ws, need);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus* status = status_of(ws);
    const int rp = jac_prec(precision), re = eloc_prec(precision);
    const bool tm = ws->timing && !graph;
    if (tm) CK(cudaEventRecord(ws->ev[0], st), "event");
    rc = run_model(md, rp, theta, configs, n_s, jb, st);
    if (rc) return rc;
    CK(launch_backward(rp, md, jb.thR, jb.Z, n_s, jb.G, st), "backward");
    CK(launch_jac_write(rp, md, jb.thR, jb.Z, jb.G, configs, n_s, O, ldo, st), "jacobian");
    if (tm) CK(cudaEventRecord(ws->ev[1], st), "event");
    if (re != rp) {
        rc = run_model(md, re, theta, configs, n_s, jbe, st);
        if (rc) return rc;
    }
    rc = run_eloc(md, re, hd, configs, n_s, jbe, eb, eloc, status, st, eloc_dp(precision, flags));
    if (rc) return rc;
    if (tm) CK(cudaEventRecord(ws->ev[2], st), "event");
    rc = run_build(O, ldo, n_s, md.n_p, nullptr, block_off, n_blocks, eloc, precision, S, F, nullptr,
                   static_cast<c128*>(Emean_out), bb, status, st, tm ? ws->ev[3] : nullptr);
    if (rc) return rc;
    // the gram stage ends (and the reduction stage starts) right before the reduction kernel
    // S comes from the library's own Gram here: the mixed solver may use the PSD certificate
    const int sv = solver == NQS_SOLVE_MIXED ? NQS_SOLVE_MIXED_PSD : solver;
    rc = run_solve(S, block_off, n_blocks, F, diag_shift, cutoff, cutoff_mode, eta, sv,
                   static_cast<c128*>(dtheta_out), evals_out, n_kept_out, a, status, st, tm ? ws->ev[5] : nullptr,
                   tm ? ws->ev[4] : nullptr, graph, step_ref_tol(precision));
    if (rc) return rc;
    if (tm) {
        CK(cudaEventRecord(ws->ev[6], st), "event");
        ws->recorded = true;
    }
    if (flags & NQS_SYNC) return nqs_sync_status(ws, stream);
    return NQS_OK;
}

// ---------------------------------------------------------------- batched step
// Several independent SR instances in one call (S9). Each instance's Jacobian, local
// energies and centring run in turn in one reused region; the split-precision operands of
// all instances go to one plane buffer (common sample stride, zero-padded: zeros add
// nothing to the Gram), so all blocks of all instances share one grouped Gram launch and
// one eigensolver launch.
namespace {

struct BatchPlan {
    long long np_tot, ns_max, ldk, sq_tot;
    int nb_tot;
    int64_t off_all[MAXB + 1];
    long long poff[MAXB + 1];  // parameter offset of each instance
    long long soff[MAXB + 1];  // S offset of each instance
    size_t inst_bytes;         // largest per-instance region
};

int plan_batch(int n_inst, const nqs_model* models, const int64_t* n_s, const nqs_hamiltonian* hams,
               const int64_t* block_off, const int32_t* n_blocks, int prec, BatchPlan* bp) {
    if (n_inst < 1 || n_inst > MAXB || !models || !n_s || !hams || !block_off || !n_blocks)
        return fail(NQS_ERR_INVALID_ARG, "sr_step_batched: bad arguments");
    if (check_prec(prec)) return NQS_ERR_INVALID_ARG;
    bp->np_tot = 0;
    bp->ns_max = 0;
    bp->sq_tot = 0;
    bp->nb_tot = 0;
    bp->inst_bytes = 0;
    bp->off_all[0] = 0;
    const int64_t* off = block_off;
    for (int i = 0; i < n_inst; ++i) {
        ModelDesc md;
        HamDesc hd;
        if (n_s[i] < 1) return fail(NQS_ERR_INVALID_ARG, "instance %d: n_s < 1", i);
        if (build_model_desc(&models[i], n_s[i], &md)) return fail(NQS_ERR_INVALID_ARG, "instance %d: bad model", i);
        if (md.kind == NQS_VIT && prec == NQS_FP32)
            return fail(NQS_ERR_UNSUPPORTED, "instance %d: the transformer runs in FP64 only", i);
        int rc = ham_desc(&hams[i], md.N, &hd);
        if (rc) return rc;
        rc = check_offsets(off, n_blocks[i], md.n_p);
        if (rc) return rc;
        if (bp->nb_tot + n_blocks[i] > MAXB)
            return fail(NQS_ERR_INVALID_ARG, "more than %d blocks over all instances", MAXB);
        bp->poff[i] = bp->np_tot;
        bp->soff[i] = bp->sq_tot;
        for (int b = 0; b < n_blocks[i]; ++b) {
            const long long n = off[b + 1] - off[b];
            bp->off_all[bp->nb_tot + b + 1] = bp->np_tot + off[b + 1];
            bp->sq_tot += n * n;
        }
        bp->nb_tot += n_blocks[i];
        bp->np_tot += md.n_p;
        bp->ns_max = n_s[i] > bp->ns_max ? n_s[i] : bp->ns_max;
        // per-instance region: model buffers, connections, O, local energies, centred e
        Arena a = sizing_arena();
        JacBufs jb, jbe;
        ElocBufs eb;
        plan_model(a, md, n_s[i], jac_prec(prec), &jb, true);
        if (eloc_prec(prec) != jac_prec(prec)) plan_model(a, md, n_s[i], eloc_prec(prec), &jbe, false);
        plan_eloc(a, md, n_s[i], hd.n_bonds, &eb);
        a.take(csize(prec) * (size_t)md.n_p * (size_t)round_up(n_s[i], 32));
        a.take(16 * (size_t)n_s[i]);
        a.take(16 * (size_t)n_s[i]);
        bp->inst_bytes = a.used > bp->inst_bytes ? a.used : bp->inst_bytes;
        off += n_blocks[i] + 1;
    }
    bp->poff[n_inst] = bp->np_tot;
    bp->soff[n_inst] = bp->sq_tot;
    bp->ldk = round_up(bp->ns_max, 64);
    return NQS_OK;
}

struct BatchBufs {
    char* inst;
    c128 *F, *S;
    void* planes[5];
    double* diag;
    int8_t* gexp;
};

void plan_batch_bufs(Arena& a, const BatchPlan& bp, int prec, BatchBufs* bb) {
    bb->inst = static_cast<char*>(a.take(bp.inst_bytes));
    bb->F = static_cast<c128*>(a.take(16 * (size_t)bp.np_tot));
    bb->S = static_cast<c128*>(a.take(16 * (size_t)bp.sq_tot));
    const int nsp = nsplit_of(prec);
    for (int q = 0; q < 5; ++q)
        bb->planes[q] = q < plane_units(nsp) ? a.take(2ull * 2 * bp.np_tot * plane_row_len(nsp, q, bp.ldk)) : nullptr;
    bb->diag = nsp ? static_cast<double*>(a.take(8 * (size_t)bp.np_tot)) : nullptr;
    bb->gexp = nsp == 5 ? static_cast<int8_t*>(a.take((size_t)(bp.ldk / GRAM_GROUP) * bp.np_tot)) : nullptr;
}

}  // namespace

extern "C" int sr_step_batched_workspace_size(int32_t n_inst, const nqs_model* models, const int64_t* n_s,
                                              const nqs_hamiltonian* hams, const int64_t* block_off,
                                              const int32_t* n_blocks, int32_t precision, size_t* bytes) {
    if (!bytes) return fail(NQS_ERR_INVALID_ARG, "bytes is NULL");
    BatchPlan* bp = new (std::nothrow) BatchPlan;
    if (!bp) return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
    int rc = plan_batch(n_inst, models, n_s, hams, block_off, n_blocks, precision, bp);
    if (!rc) {
        Arena a = sizing_arena();
        BatchBufs bb;
        plan_batch_bufs(a, *bp, precision, &bb);
        a.take(solve_workspace_bytes(bp->off_all, bp->nb_tot));
        *bytes = a.used + STATUS_BYTES;
    }
    delete bp;
    return rc;
}

extern "C" int sr_step_batched(int32_t n_inst, const nqs_model* models, const void* theta, const int8_t* configs,
                               const int64_t* n_s, const nqs_hamiltonian* hams, const int64_t* block_off,
                               const int32_t* n_blocks, double diag_shift, double cutoff, int32_t cutoff_mode,
                               double eta, int32_t precision, int32_t solver, void* dtheta_out, void* Emean_out,
                               double* evals_out, int32_t* n_kept_out, int32_t flags, nqs_workspace* ws,
                               void* stream) {
    if (!theta || !configs || !dtheta_out || !Emean_out) return fail(NQS_ERR_INVALID_ARG, "sr_step_batched: NULL");
    BatchPlan* bp = new (std::nothrow) BatchPlan;
    GramTable* tab = new (std::nothrow) GramTable;
    if (!bp || !tab) {
        delete bp;
        delete tab;
        return fail(NQS_ERR_INVALID_ARG, "host allocation failed");
    }
    int rc = plan_batch(n_inst, models, n_s, hams, block_off, n_blocks, precision, bp);
    if (rc) {
        delete bp;
        delete tab;
        return rc;
    }
    Arena a = arena_of(ws);
    BatchBufs bb;
    plan_batch_bufs(a, *bp, precision, &bb);
    Arena need = a;
    need.take(solve_workspace_bytes(bp->off_all, bp->nb_tot));
    rc = check_ws(ws, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus* status = ws ? status_of(ws) : nullptr;
    const int nsp = nsplit_of(precision);
    const int rp = jac_prec(precision), re = eloc_prec(precision);
    const char* th = static_cast<const char*>(theta);
    const int8_t* xc = configs;
    const int64_t* off = block_off;
    tab->nb = 0;
    tab->total_tiles = 0;
    for (int i = 0; i < n_inst && !rc; ++i) {
        ModelDesc md;
        HamDesc hd;
        build_model_desc(&models[i], n_s[i], &md);
        ham_desc(&hams[i], md.N, &hd);
        const long long ns = n_s[i];
        Arena ia{bb.inst, bp->inst_bytes, 0};
        JacBufs jb, jbe;
        ElocBufs eb;
        plan_model(ia, md, ns, rp, &jb, true);
        if (re != rp) plan_model(ia, md, ns, re, &jbe, false);
        else jbe = jb;
        plan_eloc(ia, md, ns, hd.n_bonds, &eb);
        const long long ldo = round_up(ns, 32);
        void* O = ia.take(csize(precision) * (size_t)md.n_p * (size_t)ldo);
        c128* eloc = static_cast<c128*>(ia.take(16 * (size_t)ns));
        c128* e = static_cast<c128*>(ia.take(16 * (size_t)ns));
        const long long po = bp->poff[i];
        rc = run_model(md, rp, th, xc, ns, jb, st);
        if (!rc) {
            cudaError_t err = launch_backward(rp, md, jb.thR, jb.Z, ns, jb.G, st);
            if (err == cudaSuccess) err = launch_jac_write(rp, md, jb.thR, jb.Z, jb.G, xc, ns, O, ldo, st);
            if (err != cudaSuccess) rc = cuda_fail(err, "jacobian");
        }
        if (!rc && re != rp) rc = run_model(md, re, th, xc, ns, jbe, st);
        if (!rc) rc = run_eloc(md, re, hd, xc, ns, jbe, eb, eloc, status, st, eloc_dp(precision, flags));
        if (!rc) {
            cudaError_t err = launch_emean(eloc, nullptr, ns, static_cast<c128*>(Emean_out) + i, e, status, st);
            void* pl[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
            for (int q = 0; q < plane_units(nsp); ++q)
                pl[q] = static_cast<__nv_bfloat16*>(bb.planes[q]) + 2 * po * plane_row_len(nsp, q, bp->ldk);
            if (err == cudaSuccess)
                err = launch_center(precision, nsp, O, ldo, ns, md.n_p, nullptr, e, bb.F + po, nullptr,
                                    nsp ? pl : nullptr, bp->ldk, nsp ? bb.diag + po : nullptr,
                                    nsp == 5 ? bb.gexp + po : nullptr, bp->np_tot, status, st);
            if (err != cudaSuccess) rc = cuda_fail(err, "centring");
        }
        // the blocks of this instance in the shared Gram table (rows and S offsets global)
        long long soff = bp->soff[i];
        for (int b = 0; b < n_blocks[i] && !rc; ++b) {
            const long long n = off[b + 1] - off[b];
            const long long T = (n + 63) / 64;
            GBlk& g = tab->b[tab->nb++];
            g.row0 = po + off[b];
            g.s_off = soff;
            g.n = (int)n;
            g.tiles = (int)(T * (T + 1) / 2);
            g.tile0 = tab->total_tiles;
            g.scale = 1.0 / (double)ns;
            tab->total_tiles += T * (T + 1) / 2;
            soff += n * n;
        }
        if (!rc && !nsp) {
            // FP64/FP32: this instance's Gram now, while its centred O is alive
            GramTable* ti = new (std::nothrow) GramTable;
            if (!ti) {
                rc = fail(NQS_ERR_INVALID_ARG, "host allocation failed");
            } else {
                gram_table(off, n_blocks[i], 64, ti);
                cudaError_t err = launch_gram_simt(precision, O, ldo, ns, nullptr, 1.0 / (double)ns, *ti,
                                                   bb.S + bp->soff[i], st);
                delete ti;
                if (err != cudaSuccess) rc = cuda_fail(err, "gram");
            }
        }
        th += 16 * (size_t)md.n_p;
        xc += (size_t)ns * md.N;
        off += n_blocks[i] + 1;
    }
    if (!rc && nsp) {
        cudaError_t err = launch_gram_tc(nsp, bb.planes, bb.gexp, bp->np_tot, 2 * bp->np_tot, bp->ldk, bp->ldk, 0.0,
                                         *tab, bb.S, status, st);
        if (err == cudaSuccess) err = launch_set_diag(bb.S, *tab, bb.diag, st);
        if (err == cudaErrorNotSupported) rc = fail(NQS_ERR_UNSUPPORTED, "tensor-core Gram needs an sm_103 device");
        else if (err != cudaSuccess) rc = cuda_fail(err, "gram");
    }
    if (!rc) {
        const int sv = solver == NQS_SOLVE_MIXED ? NQS_SOLVE_MIXED_PSD : solver;
        rc = run_solve(bb.S, bp->off_all, bp->nb_tot, bb.F, diag_shift, cutoff, cutoff_mode, eta, sv,
                       static_cast<c128*>(dtheta_out), evals_out, n_kept_out, a, status, st, nullptr, nullptr, false,
                       step_ref_tol(precision));
    }
    delete bp;
    delete tab;
    if (rc) return rc;
    if (flags & NQS_SYNC) return nqs_sync_status(ws, stream);
    return NQS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- inverse-metric diagnostics
namespace {
struct DiagPlan {
    c128 *Sa, *Sb, *Ua, *Ub;
    long long* blk_of;
    double *sig_a, *sig_b, *ev_a, *ev_b, *partial;
    void* eig;
    size_t eig_bytes;
};
void plan_diag(Arena& a, long long n, DiagPlan* d) {
    d->Sa = static_cast<c128*>(a.take(16 * (size_t)n * n));
    d->Sb = static_cast<c128*>(a.take(16 * (size_t)n * n));
    d->Ua = static_cast<c128*>(a.take(16 * (size_t)n * n));
    d->Ub = static_cast<c128*>(a.take(16 * (size_t)n * n));
    d->blk_of = static_cast<long long*>(a.take(8 * (size_t)n));
    d->sig_a = static_cast<double*>(a.take(8 * (size_t)n));
    d->sig_b = static_cast<double*>(a.take(8 * (size_t)n));
    d->ev_a = static_cast<double*>(a.take(8 * (size_t)n));
    d->ev_b = static_cast<double*>(a.take(8 * (size_t)n));
    const long long T = (n + 31) / 32;
    d->partial = static_cast<double*>(a.take(8 * (size_t)(2 + T * T)));
    d->eig_bytes = eig_vectors_workspace_bytes(n);
    d->eig = a.take(d->eig_bytes);
}
}  // namespace

extern "C" int nqs_born_weights(const void* logpsi, int64_t n, double* w_out, void* stream) {
    if (!logpsi || !w_out || n < 1) return fail(NQS_ERR_INVALID_ARG, "nqs_born_weights: bad arguments");
    CK(launch_born_weights(static_cast<const c128*>(logpsi), n, w_out, static_cast<cudaStream_t>(stream)),
       "born weights");
    return NQS_OK;
}

extern "C" int qgt_inverse_diagnostics_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 1) return fail(NQS_ERR_INVALID_ARG, "bad arguments");
    Arena a = sizing_arena();
    DiagPlan d;
    plan_diag(a, n, &d);
    *bytes = a.used + STATUS_BYTES;
    return NQS_OK;
}

extern "C" int qgt_inverse_diagnostics(const void* S_a, const int64_t* block_off_a, int32_t n_blocks_a,
                                       const void* S_b, int64_t n, double diag_shift, double cutoff,
                                       int32_t cutoff_mode, double* out, nqs_workspace* ws, void* stream) {
    if (!S_a || !S_b || !out || n < 1) return fail(NQS_ERR_INVALID_ARG, "qgt_inverse_diagnostics: bad arguments");
    if (!(diag_shift >= 0.0) || !(cutoff >= 0.0) || (cutoff_mode != 0 && cutoff_mode != 1))
        return fail(NQS_ERR_INVALID_ARG, "qgt_inverse_diagnostics: bad shift, cutoff or mode");
    int rc = check_offsets(block_off_a, n_blocks_a, n);
    if (rc) return rc;
    if (n > QL_MAXN) return fail(NQS_ERR_UNSUPPORTED, "qgt_inverse_diagnostics: n = %lld above %d", (long long)n,
                                 QL_MAXN);
    Arena a = arena_of(ws);
    DiagPlan d;
    plan_diag(a, n, &d);
    rc = check_ws(ws, a);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevStatus* status = status_of(ws);
    CK(launch_block_restrict(static_cast<const c128*>(S_a), n, block_off_a, n_blocks_a, d.Sa, d.blk_of, st),
       "block restriction");
    CK(cudaMemcpyAsync(d.Sb, S_b, 16 * (size_t)n * n, cudaMemcpyDeviceToDevice, st), "copy");
    rc = launch_eig_vectors(d.Sa, n, diag_shift, d.sig_a, d.ev_a, d.Ua, d.eig, d.eig_bytes, status, st);
    if (rc) return fail(rc, "eigen-decomposition of S_a failed");
    rc = launch_eig_vectors(d.Sb, n, diag_shift, d.sig_b, d.ev_b, d.Ub, d.eig, d.eig_bytes, status, st);
    if (rc) return fail(rc, "eigen-decomposition of S_b failed");
    CK(launch_inverse_diagnostics(n, d.sig_a, d.ev_a, d.Ua, d.sig_b, d.ev_b, d.Ub, cutoff, cutoff_mode, d.partial,
                                  out, st),
       "diagnostics");
    return NQS_OK;
}

// ---------------------------------------------------------------- build without a workspace
// qgt_block_build_static serves callers that cannot lend the library device memory (a
// plug-in interface that passes only its input and output buffers, or a process whose
// device memory another allocator holds in full). Its one scratch buffer, the centred
// local energies, is this fixed array; nothing is allocated per call.
static __device__ __align__(256) c128 g_static_e[NQS_STATIC_MAX_SAMPLES];

namespace {

constexpr int STATIC_MAX_DEVICES = 64;
std::atomic<c128*> g_static_e_addr[STATIC_MAX_DEVICES];  // device address of g_static_e, per device

// Device address of g_static_e on the current device. The address is looked up again on
// every call whose stream is not capturing (cheap), so a device reset or a re-created
// primary context cannot leave a stale address behind. During stream capture the address
// cached by the last uncaptured call on this device is used, so the first call on a device
// must come before any capture.
int static_scratch(cudaStream_t st, c128** out) {
    int dev = -1;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= STATIC_MAX_DEVICES)
        return fail(NQS_ERR_UNSUPPORTED, "device ordinal %d beyond %d", dev, STATIC_MAX_DEVICES);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap), "cudaStreamIsCapturing");
    c128* p = nullptr;
    if (cap == cudaStreamCaptureStatusNone) {
        void* q = nullptr;
        CK(cudaGetSymbolAddress(&q, g_static_e), "cudaGetSymbolAddress");
        p = static_cast<c128*>(q);
        g_static_e_addr[dev].store(p, std::memory_order_release);
    } else {
        p = g_static_e_addr[dev].load(std::memory_order_acquire);
        if (!p)
            return fail(NQS_ERR_INVALID_ARG,
                        "qgt_block_build_static: first call on device %d made during stream capture", dev);
    }
    *out = p;
    return NQS_OK;
}

}  // namespace

extern "C" int qgt_block_build_static(void* O, int64_t ldo, int64_t n_s, int64_t n_p, const double* w,
                                      const int64_t* block_off, int32_t n_blocks, const void* eloc,
                                      int32_t precision, void* S_packed, void* F_out, void* Omean_out,
                                      void* Emean_out, void* stream) {
    if (precision != NQS_FP64 && precision != NQS_FP32)
        return fail(NQS_ERR_INVALID_ARG, "qgt_block_build_static: precision %d (NQS_FP64 or NQS_FP32 only)",
                    precision);
    if (!O || !eloc || !S_packed || !F_out || n_s < 1 || n_p < 1 || ldo < n_s)
        return fail(NQS_ERR_INVALID_ARG, "qgt_block_build_static: bad arguments");
    if (n_s > NQS_STATIC_MAX_SAMPLES)
        return fail(NQS_ERR_INVALID_ARG, "qgt_block_build_static: n_s = %lld exceeds the static scratch of %d samples",
                    (long long)n_s, NQS_STATIC_MAX_SAMPLES);
    int rc = check_offsets(block_off, n_blocks, n_p);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c128* e = nullptr;
    rc = static_scratch(st, &e);
    if (rc) return rc;
    CK(launch_emean(static_cast<const c128*>(eloc), w, n_s, static_cast<c128*>(Emean_out), e, nullptr, st), "emean");
    CK(launch_center(precision, 0, O, ldo, n_s, n_p, w, e, static_cast<c128*>(F_out), static_cast<c128*>(Omean_out),
                     nullptr, 0, nullptr, nullptr, n_p, nullptr, st),
       "center");
    GramTable tab;  // host stack
    gram_table(block_off, n_blocks, 64, &tab);
    CK(launch_gram_simt(precision, O, ldo, n_s, w, w ? 1.0 : 1.0 / (double)n_s, tab, static_cast<c128*>(S_packed), st),
       "gram");
    return NQS_OK;
}
