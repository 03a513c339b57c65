// Internal descriptors and launchers shared by the translation units of libnqs_sr.
#pragma once
#include "common.cuh"

namespace nqs {

constexpr int MAXL = 32;        // max weight layers
constexpr int MAXW = 512;       // max layer width
constexpr int MAXN = 1024;      // max sites
constexpr int MAXB = 256;       // max blocks per launch table

// Network description resolved for one call (host-built, passed by value).
struct ModelDesc {
    int kind;                   // NQS_RBM / NQS_FFNN
    int L;                      // weight layers (RBM: 1)
    int N;                      // sites
    int n_p;
    int maxw;                   // max over widths (incl. N)
    int widths[MAXL + 1];
    long long woff[MAXL];       // W_l offset in theta (out x in, row-major)
    long long boff[MAXL];       // b_l offset in theta
    long long wtoff[MAXL];      // W_l^T offset in the transposed-weight copy (in x out)
    long long zoff[MAXL];       // Z_l offset in the activation store ([n_s][out_l])
    long long aoff;             // RBM visible bias offset (0)
    // transformer (NQS_VIT): patch p, tokens T = N / p, model width d, MLP width h, L encoder
    // layers; vE parameters per encoder layer; vsave saved activations per sample
    int vp, vT, vd, vh;
    long long vE, vsave;
};
// transformer limits: T <= 64, d <= 128, h <= 256, T (3 d + h) <= VIT_SMEM_CX complex values
constexpr int VIT_SMEM_CX = 6144;

int build_model_desc(const nqs_model* m, long long ns, ModelDesc* md);  // returns status
long long model_wt_elems(const ModelDesc& md);     // transposed weight copy size
long long model_z_elems(const ModelDesc& md, long long ns);

// ---- launchers (return cudaError_t of the launches) ----
// theta (c128) -> thR (cx<R>) and W^T copies
cudaError_t launch_prepare_params(int prec, const ModelDesc& md, const void* theta, void* thR,
                                  void* wtR, cudaStream_t st);
// forward: activations Z (all layers) and ln psi (c128)
cudaError_t launch_forward(int prec, const ModelDesc& md, const void* thR, const void* wtR,
                           const int8_t* x, long long ns, void* Z, c128* logpsi, cudaStream_t st);
// backward: per hidden layer G_l = dlnpsi/dz_l stored at the Z_l offsets of G
cudaError_t launch_backward(int prec, const ModelDesc& md, const void* thR, const void* Z,
                            long long ns, void* G, cudaStream_t st);
// Jacobian (parameter-major) from Z, G and x
cudaError_t launch_jac_write(int prec, const ModelDesc& md, const void* thR, const void* Z, const void* G,
                             const int8_t* x, long long ns, void* O, long long ldo, cudaStream_t st);

// ---- local energy ----
struct HamDesc {
    int n_sites, n_bonds;
    const int32_t* bond_ij;
    const double* bond_J;
    double c;
    int sign_rule;
};
// validates the bonds (0 <= i, j < n_sites, i != j): a bad bond records NQS_ERR_INVALID_ARG
// in `status` and is skipped by every later stage
cudaError_t launch_conn_count(const int8_t* x, long long ns, const HamDesc& h, int32_t* cnt, DevStatus* status,
                              cudaStream_t st);
cudaError_t launch_scan(const int32_t* cnt, long long ns, long long* off, cudaStream_t st);
cudaError_t launch_conn_fill(const int8_t* x, long long ns, const HamDesc& h, const long long* off,
                             int32_t* conn_bond, int32_t* conn_sample, cudaStream_t st);
// (hi, lo) FP32 pairs of the transposed weights (c128) for the double-float connected forwards
cudaError_t launch_split_weights(const ModelDesc& md, const void* wtR, void* wdf, cudaStream_t st);
cudaError_t launch_conn_terms(int prec, const ModelDesc& md, const void* thR, const void* wtR, const void* wdf,
                              const void* Z, const c128* logpsi, const int8_t* x, const HamDesc& h,
                              const int32_t* conn_bond, const int32_t* conn_sample,
                              const long long* nconn_ptr, long long max_conn, c128* terms, cudaStream_t st);
// FP32 difference propagation of the connected forwards (FFNN, split precisions), with the
// connections it cannot follow recomputed in double-float
struct DpBufs {
    float2* w32;                    // FP32 copy of the transposed weights [model_wt_elems]
    float4* pz;                     // (z, tanh z) of the parents' hidden units [model_z_elems]
    long long* fb_list;             // connections for the double-float kernel [max_conn]
    unsigned long long* fb_count;   // their number
};
bool dp_fallback_all();                   // test hook: every connection to the double-float kernel
int dp_width(const ModelDesc& md);        // widest hidden layer
bool dp_applicable(const ModelDesc& md);  // FFNN, >= 2 weight layers, one output, hidden width <= 512
cudaError_t launch_conn_terms_dp(const ModelDesc& md, const void* thR, const void* wtR, const void* wdf,
                                 const void* Z, const c128* logpsi, const int8_t* x, long long ns, const HamDesc& h,
                                 const int32_t* conn_bond, const int32_t* conn_sample, const long long* nconn_ptr,
                                 long long max_conn, c128* terms, const DpBufs& b, cudaStream_t st);
// ---- transformer wavefunction (vit.cu): forward with saved activations (Z: [n_s][vsave]),
// Jacobian rows (O[k * ldo + s], zero for n_s <= s < ldo), connected-configuration terms ----
cudaError_t launch_vit_forward(const ModelDesc& md, const c128* th, const int8_t* x, long long ns, c128* Z,
                               c128* logpsi, cudaStream_t st);
cudaError_t launch_vit_jacobian(const ModelDesc& md, const c128* th, const c128* Z, const int8_t* x, long long ns,
                                c128* O, long long ldo, cudaStream_t st);
cudaError_t launch_vit_conn_terms(const ModelDesc& md, const c128* th, const c128* logpsi, const int8_t* x,
                                  const HamDesc& h, const int32_t* conn_bond, const int32_t* conn_sample,
                                  const long long* nconn_ptr, long long max_conn, c128* terms, cudaStream_t st);

// ---- exchange-move Metropolis sampler and parameter update (sampler.cu) ----
cudaError_t launch_mc_setup(long long n, double* bond_J, int32_t* csamp, int32_t* cbond, long long* nconn,
                            cudaStream_t st);
cudaError_t launch_mc_propose(const int8_t* x, int N, long long n, const double* u, int32_t* pairs, int32_t* valid,
                              cudaStream_t st);
cudaError_t launch_mc_accept(int8_t* x, int N, long long n, const double* u, const int32_t* pairs,
                             const int32_t* valid, const c128* ratio, unsigned long long* n_acc, cudaStream_t st);
cudaError_t launch_theta_update(c128* theta, const c128* dtheta, long long n, cudaStream_t st);
cudaError_t launch_eloc_reduce(const int8_t* x, long long ns, const HamDesc& h,
                               const long long* off, const c128* terms, c128* eloc,
                               DevStatus* status, cudaStream_t st);

// ---- centring / force ----
cudaError_t launch_emean(const c128* eloc, const double* w, long long ns, c128* emean, c128* e,
                         DevStatus* status, cudaStream_t st);
// nsplit 0: dO written in place (prec FP64/FP32); nsplit 2 or 3: element-wise BF16
// split planes of dO (O is c128, unchanged)
// (split modes also write diag[k] = sum_s w_s |dO_k(s)|^2 in FP64; nsplit 5 = grouped
// error-free split with int8 exponents gexp[group][param], groups of GRAM_GROUP samples,
// stored as three plane units, see plane_units)
cudaError_t launch_shard_sums(int prec, const void* O, long long ldo, long long ns, long long np, const c128* eloc,
                              c128* osum, c128* esum, cudaStream_t st);
cudaError_t launch_ecenter(const c128* eloc, long long ns, const c128* emean, c128* e, cudaStream_t st);
// means[0..np) = osum / n_total, means[np] = esum[0] / n_total (global means of a sharded step)
cudaError_t launch_sums_to_means(const c128* osum, const c128* esum, long long np, long long n_total, c128* means,
                                 cudaStream_t st);
// sample-major grouped split of a centred block (c128 dO [nb][ldo]) for the sample-space Gram:
// planes[q] rows 2s, 2s+1 along ldk (multiple of 64) parameters, gexp[k / GRAM_GROUP][s],
// diag[s] = sum_k |dO_k(s)|^2 / ns
cudaError_t launch_transpose_group(const c128* dO, long long ldo, long long ns, long long nb, void* const* planes,
                                   int8_t* gexp, long long ldk, double* diag, cudaStream_t st);
// sample-space (NTK) comparator
cudaError_t launch_ntk_transpose(int prec, const c128* O, long long ldo, long long ns, long long np, void* Y,
                                 long long ldy, cudaStream_t st);
cudaError_t launch_ntk_rhs(const c128* e, long long ns, c128* rhs, cudaStream_t st);
cudaError_t launch_ntk_back(const c128* O, long long ldo, long long ns, long long np, const c128* u, double eta,
                            c128* dtheta, cudaStream_t st);
cudaError_t launch_vjp(int prec, const void* O, long long ldo, long long ns, long long np, const c128* g, c128* out,
                       cudaStream_t st);
cudaError_t launch_center(int prec, int nsplit, void* O, long long ldo, long long ns, long long np,
                          const double* w, const c128* e, c128* F, c128* Omean, void* const* planes, long long ldk,
                          double* diag, int8_t* gexp, long long gstride, DevStatus* status, cudaStream_t st,
                          const c128* mean_in = nullptr, double wconst = 0.0);

// ---- Gram ----
struct GBlk {                   // one QGT block of one instance
    long long row0;             // first parameter row of the block in the operand
    long long s_off;            // first element of S_b in the packed output
    int n;                      // block size
    int tiles;                  // lower-triangle tile count
    long long tile0;            // prefix of tiles over previous blocks
    double scale;               // 1/N_s of the block's instance; 0: the launch's scale
};
struct GramTable {
    int nb;
    int group;                  // tensor-core Gram: edge of the square groups of tiles taken in turn (1: by rows)
    long long total_tiles;
    GBlk b[MAXB];
};
// Tile-group edge of the tensor-core Gram for a call whose largest block has max_nb parameters
// and which sums ns samples: the tuning table's first matching entry (nqs_set_gram_tuning),
// else GRAM_GROUP_EDGE_DEFAULT.
constexpr int GRAM_GROUP_EDGE_DEFAULT = 8;
int gram_group_edge(long long max_nb, long long ns);
cudaError_t launch_gram_simt(int prec, const void* dO, long long ldo, long long ns, const double* w,
                             double scale, const GramTable& tab, c128* S, cudaStream_t st);
constexpr int GRAM_KPI_DEFAULT = 4;    // MMA K-steps (16 samples) per accumulator flush
constexpr int GRAM_GROUP = 32;         // samples per exponent group of the grouped split (gexp rows)
// Storage of the split planes: nsplit arrays of 2 np rows x ldk BF16 for the element-wise
// splits; for the grouped five-slice split three units: slices 1-2 and slices 3-4 each share
// rows of 2 ldk (group g of slice 2u + h at columns 64 g + 32 h .. + 31, so that one 128-byte
// row of the tensor-core Gram's TMA boxes carries two slices of a group), slice 5 alone in
// rows of ldk.
inline int plane_units(int nsplit) { return nsplit == 5 ? 3 : nsplit; }
inline long long plane_row_len(int nsplit, int unit, long long ldk) {
    return (nsplit == 5 && unit < 2) ? 2 * ldk : ldk;
}
// tcgen05 Gram over nsplit element-wise BF16 split planes (2: 3 products; 3: 6 products),
// FP32 accumulation per 64-sample K block folded into double-float sums;
// cudaErrorNotSupported off sm_103.
cudaError_t launch_gram_tc(int nsplit, const void* const* planes, const int8_t* gexp, long long np, long long rows,
                           long long ldk, long long kpad, double scale, const GramTable& tab, c128* S,
                           DevStatus* status, cudaStream_t st);
void gram_table(const int64_t* block_off, int nb, int tile_rows, GramTable* tab);
// overwrite the diagonal of every S_b with diag (FP64 sums of |dO_k|^2)
cudaError_t launch_set_diag(c128* S, const GramTable& tab, const double* diag, cudaStream_t st);

// ---- iteration limits and device wait budget ----
// Defaults: 60 implicit-QL sweeps per eigenvalue, 30 refinement sweeps, 2 s per device-side
// wait. nqs_set_limits (a test hook) lowers them so that the failure paths can be driven
// on purpose: a limit that runs out records NQS_ERR_NOT_CONVERGED or NQS_ERR_TIMEOUT.
struct Limits {
    int ql_maxit;
    int ref_maxit;
    unsigned long long wait_ns;
};
Limits limits();

// ---- per-block solve ----
struct SolveArgs {
    double shift, cutoff, eta;
    int cutoff_mode;
    bool want_evals;
    bool mixed;                 // FP32 reduction + FP64 iterative refinement
    bool psd;                   // S_b is a Gram matrix: sigma_min >= shift - 1e-6 sigma_max
    cudaEvent_t ev_trd_done;    // recorded after the tridiagonal reduction (or NULL)
    cudaEvent_t ev_trd_start;   // recorded just before the tridiagonal reduction (or NULL)
    bool no_host_sync;          // capturable: the mixed certificate is checked on the device
    int ql_maxit;               // implicit-QL sweep limit per eigenvalue
    bool want_vectors;          // FP64 path: form every block's tridiagonal eigenvectors (QL)
    double ref_tol = 1e-14;     // Cholesky path: refine until ||r|| <= ref_tol ||F|| (or the floor)
};
size_t solve_workspace_bytes(const int64_t* block_off, int nb);
// Full FP64 eigen-decomposition of one n x n Hermitian matrix S (lower triangle used;
// OVERWRITTEN with reflectors): S + shift I = U diag(sig) U^H. sig[i] (unsorted) pairs with
// the eigenvector U[i*n .. i*n+n) (eigenvector-major); evals_asc gets the eigenvalues ascending.
size_t eig_vectors_workspace_bytes(long long n);
int launch_eig_vectors(c128* S, long long n, double shift, double* sig, double* evals_asc, c128* U, void* work,
                       size_t work_bytes, DevStatus* status, cudaStream_t st);
// Inverse-metric diagnostics (Eq. 4) from two eigen-decompositions (diagnostics.cu)
cudaError_t launch_born_weights(const c128* logpsi, long long n, double* w, cudaStream_t st);
cudaError_t launch_block_restrict(const c128* S, long long n, const int64_t* block_off, int nb, c128* out,
                                  long long* blk_of, cudaStream_t st);
cudaError_t launch_inverse_diagnostics(long long n, const double* sig_a, const double* ev_a, const c128* Ua,
                                       const double* sig_b, const double* ev_b, const c128* Ub, double cutoff,
                                       int mode, double* partial, double* out, cudaStream_t st);
int launch_block_solve(c128* S, const int64_t* block_off, int nb, const c128* F,
                       const SolveArgs& a, c128* dtheta, double* evals, int32_t* n_kept,
                       void* work, size_t work_bytes, DevStatus* status, cudaStream_t st);

}  // namespace nqs
