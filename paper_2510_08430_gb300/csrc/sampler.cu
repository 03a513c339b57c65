// Exchange-move Metropolis sampling of |psi|^2 (Markov-chain sampling of the VMC loop, Sec. 1)
// and the parameter update theta <- theta + dtheta (Sec. 2).
//
// One step gives every chain one proposal: the k1-th up spin i (k1 = floor(u1 n_up)) and the
// k2-th down spin j (k2 = floor(u2 n_down)), counted in site order, are exchanged, which keeps
// total S^z; the move is accepted when u3 < |psi(x') / psi(x)|^2. The proposal is symmetric,
// so the chains sample |psi|^2 in their S^z sector. The ratio psi(x')/psi(x) is exactly the
// connected-configuration ratio of the local energies (spins i and j flipped), so the step
// reuses the FP64 connected forwards of eloc.cu with the proposals as a one-bond-per-chain
// table (coupling 1/2, c = 1, no sign rule: the "term" is then the ratio itself).
#include "internal.cuh"

namespace nqs {

// bond table of the proposals: chain c's pair at pairs[2c], coupling 1/2, connection c = (c, c)
__global__ void mc_setup_kernel(long long n, double* __restrict__ bond_J, int32_t* __restrict__ csamp,
                                int32_t* __restrict__ cbond, long long* __restrict__ nconn) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        bond_J[c] = 0.5;
        csamp[c] = (int32_t)c;
        cbond[c] = (int32_t)c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *nconn = n;
}

// pairs[2c], pairs[2c+1] = (i, j) of chain c; valid[c] = 0 when the chain has no up or no
// down spin (the pair is then (0, 0 or 1), in range, and never accepted)
__global__ void mc_propose_kernel(const int8_t* __restrict__ x, int N, long long n, const double* __restrict__ u,
                                  int32_t* __restrict__ pairs, int32_t* __restrict__ valid) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int8_t* row = x + c * N;
        int n_up = 0;
        for (int s = 0; s < N; ++s) n_up += row[s] == 1 ? 1 : 0;
        const int n_dn = N - n_up;
        const double* uc = u + 3 * c;
        int i = 0, j = N > 1 ? 1 : 0, ok = 0;
        if (n_up > 0 && n_dn > 0) {
            int k1 = (int)floor(uc[0] * (double)n_up), k2 = (int)floor(uc[1] * (double)n_dn);
            k1 = k1 < n_up ? k1 : n_up - 1;  // u < 1; guards a caller's u = 1
            k2 = k2 < n_dn ? k2 : n_dn - 1;
            for (int s = 0; s < N; ++s) {
                if (row[s] == 1) {
                    if (k1-- == 0) i = s;
                } else {
                    if (k2-- == 0) j = s;
                }
            }
            ok = 1;
        }
        pairs[2 * c] = i;
        pairs[2 * c + 1] = j;
        valid[c] = ok;
    }
}

// accept when u3 < |ratio|^2; an accepted move flips spins i and j of the chain
__global__ void mc_accept_kernel(int8_t* __restrict__ x, int N, long long n, const double* __restrict__ u,
                                 const int32_t* __restrict__ pairs, const int32_t* __restrict__ valid,
                                 const c128* __restrict__ ratio, unsigned long long* __restrict__ n_acc) {
    unsigned long long a = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        if (!valid[c]) continue;
        const c128 r = ratio[c];
        if (u[3 * c + 2] < r.re * r.re + r.im * r.im) {
            int8_t* row = x + c * N;
            row[pairs[2 * c]] = (int8_t)(-row[pairs[2 * c]]);
            row[pairs[2 * c + 1]] = (int8_t)(-row[pairs[2 * c + 1]]);
            ++a;
        }
    }
    if (n_acc) {
        a = warp_sum(a);
        if ((threadIdx.x & 31) == 0 && a) atomicAdd(n_acc, a);
    }
}

__global__ void theta_update_kernel(c128* __restrict__ theta, const c128* __restrict__ dtheta, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        theta[k] = theta[k] + dtheta[k];
}

static unsigned grid_for(long long n) {
    const long long g = (n + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

cudaError_t launch_mc_setup(long long n, double* bond_J, int32_t* csamp, int32_t* cbond, long long* nconn,
                            cudaStream_t st) {
    count_launch();
    mc_setup_kernel<<<grid_for(n), 256, 0, st>>>(n, bond_J, csamp, cbond, nconn);
    return cudaGetLastError();
}
cudaError_t launch_mc_propose(const int8_t* x, int N, long long n, const double* u, int32_t* pairs, int32_t* valid,
                              cudaStream_t st) {
    count_launch();
    mc_propose_kernel<<<grid_for(n), 256, 0, st>>>(x, N, n, u, pairs, valid);
    return cudaGetLastError();
}
cudaError_t launch_mc_accept(int8_t* x, int N, long long n, const double* u, const int32_t* pairs,
                             const int32_t* valid, const c128* ratio, unsigned long long* n_acc, cudaStream_t st) {
    count_launch();
    mc_accept_kernel<<<grid_for(n), 256, 0, st>>>(x, N, n, u, pairs, valid, ratio, n_acc);
    return cudaGetLastError();
}
cudaError_t launch_theta_update(c128* theta, const c128* dtheta, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    theta_update_kernel<<<grid_for(n), 256, 0, st>>>(theta, dtheta, n);
    return cudaGetLastError();
}

}  // namespace nqs
