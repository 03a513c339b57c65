// Shared definitions of the per-block eigensolver (eigh.cu) and of its persistent,
// grid-synchronised kernels (eigh_persist.cu).
#pragma once
#include "internal.cuh"

namespace nqs {

constexpr int TB = 64;       // tile of the fused update + matvec
constexpr int CH = 256;      // rows per CTA in the vector kernels
constexpr int MAXCH = 512;   // max row chunks per block (n <= 131072)
constexpr int DCH = 32;      // rows per unit of the tile-partial reductions
constexpr int MAXDCH = MAXCH * (CH / DCH);
constexpr int QL_MAXN = 12000;

struct EBlk {
    long long off;    // offset of the block in length-n_p arrays
    long long soff;   // offset of S_b in the packed matrix array
    long long yoff;   // offset of the block's matvec partials
    int n;
    int T;            // ceil(n / TB)
    int orig;         // index of the block in the caller's order
    int pad;
};
struct EBTab {
    int nb;
    EBlk b[MAXB];
};
struct BlkInfo {
    double sigma_max;
    double thr;
    int n_dropped;
    int n_kept;
};

struct SolveBufs {
    const EBlk* tab;
    unsigned* bar;        // grid-barrier state of the persistent kernels (2 words)
    c128* S;
    double *d, *e, *e2, *ev;
    c128 *tau, *f, *v0, *v1, *w, *x, *z;
    BlkInfo* info;
    c128* bcol;          // column buffer of the reduction (c64 view in the FP32 reduction)           // column-norm partials of the reduction [nb][MAXDCH][2]
    c128 *pvf, *pxv, *ypart;
    double* zmat;
};

// Views used by the Householder reduction in precision R (FP64 exact path,
// FP32 preconditioner of the mixed path). f == nullptr skips the Q^H F update.
template <typename R> struct TrdBufs {
    const EBlk* tab;
    cx<R>* A;
    cx<R> *v0, *v1, *w, *x, *ypart;
    c128* f;
    double *d, *e, *e2;
    c128 *tau, *pvf, *pxv;
    cx<R>* bcol;          // next column, updated except for the alpha part of the last reflector
};

constexpr int QNB = 32;      // reflectors per panel of the blocked (WY) application of Q
constexpr double REF_TOL = 1e-14;
constexpr double REF_FLOOR = 1e-12;  // accepted once the residual stops contracting (rounding floor)

struct MixBufs {
    const EBlk* tab;
    const c128* S;        // FP64 S (lower triangles), packed
    c64* Sf;              // FP32 copy, reduced in place (reflectors in the upper rows)
    c64* Tf;              // T factors: per block ceil((n-1)/QNB) panels x QNB x QNB
    long long* toff;      // per slot offset into Tf
    c64* pdot;            // panel dot products V_p^H y: [2][sum of row chunks][QNB]
    double *d, *e;        // FP32-reduced tridiagonal (stored in FP64)
    double *piv, *lmul;   // LDL^T of T + lambda I
    float *ds32, *e232;   // FP32 d + lambda and e^2 for the certificate's Sturm counts
    c128 *x, *r;          // refinement iterate and residual (FP64)
    c64 *r32, *y32, *w32; // FP32 work vectors
    c128* hpart;          // FP64 Hermitian matvec partials (T^2 x 64 per block)
    double* rn;           // per slot ||r||^2 partials [MAXCH]
    double* fn;           // per slot ||F||^2
    int* done;            // per slot converged flag
    int* fallback;        // per slot: cutoff may drop an eigenvalue (needs the FP64 path)
};

// Cholesky path for Gram-matrix blocks (chol.cu): certificate from ||S_b||_F, FP32 tiled
// Cholesky of S_b + lambda I, FP64-residual refinement. Blocks of at most 65536 parameters.
bool chol_applicable(const int64_t* block_off, int nb);
size_t chol_workspace_bytes(const int64_t* block_off, int nb);
// Writes dtheta and n_kept when every block succeeds. *ok_out (host): every block certified,
// factored and converged (always true under capture, where a failure is NQS_ERR_RETRY).
int launch_chol_solve(const c128* S, const int64_t* block_off, int nb, const c128* F, const SolveArgs& a,
                      c128* dtheta, int32_t* n_kept, void* work, size_t work_bytes, DevStatus* status,
                      cudaStream_t st, bool* ok_out);

// Persistent cooperative kernels (eigh_persist.cu). `bar` points to two zeroed words
// of grid-barrier state; every grid-wide wait is bounded and reports NQS_ERR_TIMEOUT.
template <typename R>
int launch_trd_persist(const TrdBufs<R>& B, const EBTab& tab, unsigned* bar, DevStatus* status, cudaStream_t st);
int launch_refine_persist(const SolveBufs& B, const MixBufs& M, const EBTab& tab, const c128* F, double shift,
                          unsigned* bar, DevStatus* status, cudaStream_t st);

}  // namespace nqs
