// Problems (2) and (3) of Section 4.2 around the momentum solve.
//
// With the ALE derivatives dropped (Eq. (REDUCEDMATRIX)) the Newton step of a
// time step is three sub-steps in order: problem (1), the condensed momentum
// system for the velocity and pressure updates; problem (2), the discrete
// zero-order relation between deformation and velocity on the interface and in
// the solid, whose Newton step carries the mass matrix on both sides and is
// therefore one vector addition, du = r + k theta dv (velocity components, on
// the nodes of solid cells); problem (3), the extension of the deformation
// into the fluid, E_ff du_f = b_5 - E_fi du_i, whose right-hand side lifts the
// deformation now known on the fixed nodes through the coupling of the
// extension operator as assembled (before its fixed rows and columns are
// reduced to the identity).
#include "elem.cuh"

namespace nmg {

namespace {

using namespace elem;

// du_i = r_i + k_theta (dv_i)_{0..DIM-1} on flagged nodes, 0 elsewhere.
template <int DIM>
__global__ void __launch_bounds__(256) k_deformation_update(int64_t nodes, const double* __restrict__ r,
                                                             const double* __restrict__ dv, double k_theta,
                                                             const uint8_t* __restrict__ update_nodes,
                                                             double* __restrict__ du) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nodes) return;
    const bool on = update_nodes[i] != 0;
    double v[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) v[c] = on ? fma(k_theta, dv[i * (DIM + 1) + c], r[i * DIM + c]) : 0.0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) du[i * DIM + c] = v[c];
}

// rhs = g on fixed unknowns, b5 - E g_hat on free ones (g_hat = g on the fixed
// unknowns and 0 elsewhere; E the unreduced extension operator in stencil
// layout, FP64).  One thread per node, the stencil terms in the order of every
// other product of the library.
template <int DIM>
__global__ void __launch_bounds__(256) k_extension_rhs(Geom g, const double* __restrict__ E,
                                                       const uint8_t* __restrict__ fixed,
                                                       const double* __restrict__ b5, const double* __restrict__ gv,
                                                       double* __restrict__ rhs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.nodes) return;
    double acc[DIM];
    auto ghat = [&](int64_t j, int, int, int, double* xv) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) xv[c] = fixed[j * DIM + c] ? gv[j * DIM + c] : 0.0;
    };
    spmv_acc_f<double, DIM, decltype(ghat)&, true, 1, DIM>(g, E, ghat, i, acc);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const int64_t k = i * DIM + c;
        rhs[k] = fixed[k] ? gv[k] : b5[k] - acc[c];
    }
}

}  // namespace

void launch_deformation_update(int dim, int64_t nodes, const double* r, const double* dv, double k_theta,
                               const uint8_t* update_nodes, double* du, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid((unsigned)((nodes + 255) / 256)), block(256);
    if (dim == 2) k_deformation_update<2><<<grid, block, 0, s>>>(nodes, r, dv, k_theta, update_nodes, du);
    else k_deformation_update<3><<<grid, block, 0, s>>>(nodes, r, dv, k_theta, update_nodes, du);
}

void launch_extension_rhs(const Geom& g, const double* E, const uint8_t* fixed, const double* b5, const double* gv,
                          double* rhs, cudaStream_t s) {
    g_launches += 1;
    const dim3 grid((unsigned)((g.nodes + 255) / 256)), block(256);
    if (g.dim == 2) k_extension_rhs<2><<<grid, block, 0, s>>>(g, E, fixed, b5, gv, rhs);
    else k_extension_rhs<3><<<grid, block, 0, s>>>(g, E, fixed, b5, gv, rhs);
}

}  // namespace nmg
