// Internal data structures shared by the kernels and the host orchestration.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "smc.h"

#define SMC_MAX_NS 64
#define SMC_MAX_SIDE 4        // species per reaction side
#define SMC_GHOST 4           // ghost cells per side (8th-order stencils)
#define SMC_EXP_TABLE 2048    // entries of the exponential's 2^(j/N) table

namespace smc {

constexpr double kRu = 8.31446261815324e7;     // erg/(mol K)
constexpr double kRc = 1.98720425864083;       // cal/(mol K)
constexpr double kPatm = 1.01325e6;            // dyn/cm^2

// Device-resident mechanism tables (one per handle).
struct Mech {
  int ns, nr;
  double Ru_W[SMC_MAX_NS];        // R_u / W_k
  double W[SMC_MAX_NS];
  double invW[SMC_MAX_NS];
  double invLe[SMC_MAX_NS];
  double cp[SMC_MAX_NS][5];       // cp/R = c0 + c1 T + ... + c4 T^4
  double hT[SMC_MAX_NS][6];       // h/R  = a6 + T (a1 + T (a2/2 + ...))
  double sR[SMC_MAX_NS][6];       // s/R  = a1 ln T + a7 + T (a2 + T (a3/2 + ...)) : {a1, a7, a2, a3/2, a4/3, a5/4}
  double gW[SMC_MAX_NS][7];       // g/RT - ln W_k = a6/T + (a1 - a7 - ln W_k) - a1 ln T
                                  //   + T (-a2/2 + T (-a3/6 + T (-a4/12 + T (-a5/20))))
                                  //   : {a6, a1 - a7 - ln W_k, -a1, -a2/2, -a3/6, -a4/12, -a5/20}
  double eta_ref, inv_T_ref, eta_exp, inv_Pr;
  double inv_ns;
  int alu;                        // rate arithmetic moved off the FP64 pipe (SMC_OPT_ALU): 1 the
                                  // exponentials (exp_alu), 2 also the products (dmul_alu)
  double exp2tab[SMC_EXP_TABLE];  // 2^(j/2048) (table of fast_exp and exp_alu)
  float exp2tabf[SMC_EXP_TABLE];  // the same rounded to float (mixed-precision rates)
  // float copies for the mixed-precision transport (no conversions in kernels)
  float hTf[SMC_MAX_NS][6];
  float Ru_Wf[SMC_MAX_NS];
  float invLef[SMC_MAX_NS];
  float eta_ref_f, inv_T_ref_f, eta_exp_f, inv_Pr_f;
};

struct Reaction {
  double lnA;                     // ln A - sum_k nu'_k ln W_k
  double b, Ea_R;                 // temperature exponent; Ea / R_c (K)
  double fcd[SMC_MAX_SIDE];       // nu'_k as doubles (no int->double conversions)
  double fcw[SMC_MAX_SIDE];       // nu' W_k and nu'' W_k: production rates in g/(cm^3 s)
  double rcw[SMC_MAX_SIDE];       //   accumulate without a final multiply
  float fcwf[SMC_MAX_SIDE];       // the same as floats (mixed-precision rates)
  float rcwf[SMC_MAX_SIDE];
  int nf, nr_;                    // species on each side
  int fk[SMC_MAX_SIDE];
  int rk[SMC_MAX_SIDE];
  int fm[3], rm[3];               // the molecules of each side (species repeated nu times)
  int nfm, nrm;
  int dn;                         // sum_k nu''_k - nu'_k, -3..3
  int pad;
};

// Pack and check a mechanism; nullptr on success, else the reason.
const char *pack_mechanism(const smc_mechanism *mech, int max_reactions, Mech &M,
                           std::vector<Reaction> &rx);

// Geometry of one box in the ghosted (Q) and interior (U) layouts.
struct Box {
  int nx, ny, nz;
  int gx, gy, gz;                 // ghosted extents n + 8
  long long off_g, off_i;         // first ghosted / interior cell
  int lo[3];                      // global index of the first interior cell
  int pad;
};

// An interior cell within four cells of a non-periodic x end: its x-direction
// terms use the boundary-lowered stencils (Sec. 2.2, boundary paragraph).
struct BcCell {
  long long g, i;                 // ghosted and interior index
  int k;                          // distance from the end, 0..3
  int side;                       // 0: low x end, 1: high x end
};

// One thread's share of a stencil direction: a segment of one grid line.
struct LineItem {
  long long g0;                   // ghosted index of the first cell of the segment
  long long i0;                   // interior index of that cell
  int sg, si;                     // strides along the line (ghosted, interior)
  int len;                        // cells in the segment
  int pad;
};

// Runtime options passed to the kernels by value.
struct Opts {
  int mode;                       // 0 correction velocity, 1 reference species
  int ref;
  int reactions;
  int maxit;
  int rates32;                    // 1: production rates with FP32 mantissas (mixed precision only)
  int chain_blocks;               // cap on resident reaction-chain blocks per SM (0: none)
  int persistent;                 // 1: resident-capacity grids that loop over their work items
  double tol, T0, xi_ratio;
};

// Stencil coefficients, per direction, scaled by 1/h^2 (narrow) or 1/h (D).
struct Coef {
  double M[3][8][8];
  double D[3][4];
  double S[8];                    // unused padding for alignment
};

// Q field indices (ghosted primitive / coefficient scratch).
enum {
  Q_U = 0, Q_V, Q_W, Q_T, Q_P, Q_RHO, Q_RHOH, Q_C43, Q_ETA, Q_C23, Q_LAM,
  Q_HMIX, Q_AP, Q_SB, Q_KX, Q_KY, Q_KZ, Q_NBASE
};
// float-plane indices of the mixed-precision scratch (reuses the FP64 Q buffer)
enum {
  PM_U = 0, PM_V = 2, PM_W = 4, PM_T = 6, PM_P = 8, PM_KX = 10, PM_KY = 12, PM_KZ = 14,
  PM_HMIX = 16, PM_RHO = 18, PM_RHOH = 20,
  PM_C43 = 22, PM_ETA, PM_C23, PM_LAM, PM_AP, PM_SB, PM_NBASE
};
__host__ __device__ inline int pmY(int ns, int k) { return PM_NBASE + 2 * k; }
__host__ __device__ inline int pmX(int ns, int k) { return PM_NBASE + 2 * ns + 2 * k; }
__host__ __device__ inline int pmRY(int ns, int k) { return PM_NBASE + 4 * ns + 2 * k; }
__host__ __device__ inline int pmRD(int ns, int k) { return PM_NBASE + 6 * ns + k; }
__host__ __device__ inline int pmRDH(int ns, int k) { return PM_NBASE + 7 * ns + k; }
__host__ __device__ inline int pmB(int ns, int k) { return PM_NBASE + 8 * ns + k; }
// species blocks start at Q_NBASE: Y, X, rhoY, rhoD, rhoD*h', B
inline __host__ __device__ int qY(int ns) { return Q_NBASE; }
inline __host__ __device__ int qX(int ns) { return Q_NBASE + ns; }
inline __host__ __device__ int qRY(int ns) { return Q_NBASE + 2 * ns; }
inline __host__ __device__ int qRD(int ns) { return Q_NBASE + 3 * ns; }
inline __host__ __device__ int qRDH(int ns) { return Q_NBASE + 4 * ns; }
inline __host__ __device__ int qB(int ns) { return Q_NBASE + 5 * ns; }
inline __host__ __device__ int nQ(int ns) { return Q_NBASE + 6 * ns; }

// Device status bits.
enum : unsigned { ST_NONCONV = 1u, ST_NONPHYS = 2u, ST_NONFINITE = 4u };

// Host-side quadrature (Gauss-Lobatto nodes, Lagrange integration matrices).
void narrow8_matrix(double m47, double m48, double M[8][8]);
void lobatto_nodes(int n, std::vector<double> &x);
void node_to_node_matrix(const std::vector<double> &nodes, std::vector<double> &S);
void multirate_matrices(int coarse, int fine, int repeat, std::vector<double> &t1,
                        std::vector<double> &t2, std::vector<double> &S21,
                        std::vector<double> &S22);

// Kernel launchers (kernels_*.cu).
struct DevState {
  int ns, nv, nq, nboxes;
  long long ncells, nghost;
  const Mech *mech;
  const Reaction *rx;
  const Coef *hcoef;               // host copy (read by the launchers only)
  const Box *boxes;
  const int *gmap;                // ghosted cell -> interior index of its periodic image
  const long long *imap;          // interior cell -> ghosted index
  const LineItem *lines[3];
  long long nlines[3];
  double *Q;                      // [nq][nghost]
  double *G;                      // [9][nghost] velocity gradients D_e u_c
  double *Qt, *Gt;                // the same fields with x the slowest index in each box
  const long long *xt_tiles;      // [nboxes + 1] prefix of 32x32 (x, y) tiles per box
  double *divacc;                 // [ncells] sum_k narrow species divergence
  unsigned *status;
  Opts opt;
  float xi_ratio_f;
  int x_outflow;                  // 1: the x ends are non-periodic boundaries
  int nx_domain;                  // cells of the domain along x
  const BcCell *bc_cells;         // the cells next to the x ends (x_outflow only)
  long long n_bc;
  const long long *halo_dst;      // ghost cells (ghosted index) ...
  const long long *halo_src;      // ... and the ghosted index of their periodic image
  long long nhalo;                // 0: primitives are evaluated at every ghosted cell
  int warm_T;                     // 1: the mixed primitive planes hold the temperatures of an
                                  //    earlier evaluation (first guess of the Newton solve)
};

// Boundary-lowered x-direction terms at the cells next to the x ends; they
// replace what the x line kernel stored there (FP64 result, or the float
// accumulator of the mixed path).  Launch after the x-direction line kernel
// and before the y and z ones.
void launch_xbc(const DevState &s, double *dU, cudaStream_t st);
void launch_xbc_m(const DevState &s, float *dUf, cudaStream_t st);

// Blocks of `threads` threads and `smem` bytes of dynamic shared memory that
// the current device holds at once for kernel f (occupancy calculator x SM
// count), cached per device in *cache (an array of 64, zero-initialised) on
// the first (eager) launch, before any stream capture.
template <typename K>
int resident_blocks(K f, int threads, size_t smem, int *cache) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, smem);
    cache[dev] = per * sms > 0 ? per * sms : 1;
  }
  return cache[dev];
}

// Primitives at every ghosted cell, each through the gather map (no halo list needed).
void launch_prim(const DevState &s, const double *U, cudaStream_t st);
// Primitives at the interior cells only, then launch_halo.
void launch_prim_interior(const DevState &s, const double *U, cudaStream_t st);
// Fill the ghost cells of `planes` primitive planes (element size 8 or 4)
// from their periodic images through the halo list (s.nhalo entries).
void launch_halo(const DevState &s, int planes, int esize, cudaStream_t st);
void launch_grad(const DevState &s, cudaStream_t st);
void launch_march(const DevState &s, int dir, double *dUdt, int first, cudaStream_t st);
// FP64 sliding-window line kernel (variant 1: 16-cell chunks, 2: 32-cell chunks,
// 3: 8-cell chunks with the pressure products of every face kept in shared memory)
void launch_march_w(const DevState &s, int dir, double *dUdt, int first, int variant,
                    cudaStream_t st);
void launch_final(const DevState &s, double *dUdt, int transport, int chemistry, cudaStream_t st);
void launch_prim_to_cons(const DevState &s, const double *prim, double *U, cudaStream_t st);
// Copy `planes` planes of element size `esize` (4 or 8) from the box layout
// [z][y][x] to [x][z][y] per ghosted box (for the x-direction stencil march).
void launch_transpose_x(const DevState &s, const void *src, void *dst, int planes, int esize,
                        cudaStream_t st);

// Mixed precision (kernels_mixed.cu): FP32 stencils / transport on float-pair
// scratch in the Q buffer, FP64 temperature, chemistry and accumulation.
int nQm(int ns);
void launch_prim_m(const DevState &s, const double *U, cudaStream_t st);
void launch_grad_m(const DevState &s, cudaStream_t st);
// variant 1: 16-cell chunks, 3 blocks/SM; 2: 32-cell chunks, 3 blocks/SM;
// 3: 16-cell chunks, 4 blocks/SM
void launch_march_m2(const DevState &s, int dir, float *dUf, int first, int variant,
                     cudaStream_t st);
void launch_final_m(const DevState &s, const double *U, const float *dUf, double *dU, int transport,
                    int chemistry, cudaStream_t st);

// out = in + sum_i c[i] * src[i] over n doubles (in may be null: zero)
struct Combo {
  int nsrc;
  double c[12];
  const double *src[12];
};
void launch_combo(const double *in, double *out, const Combo &cb, long long n, cudaStream_t st);

// Multirate fine-node chain over one coarse interval (eq. mrupdate).  Fine
// substeps q = q0 .. q0+nsub-1 lie in one Gauss-Lobatto group whose nodes are
// q0 .. q0+nsub (type (b): one group per coarse interval).
struct FineChain {
  int q0, nsub, p, M1;
  double dtq[8];                  // dt * (t2[q+1] - t2[q])
  double s21[8][5];               // dt * S21[q][j] - [j == p] dtq: coarse-node weights with the
                                  //   -dtq f1(U^k_p) correction term folded in
  double s22[8][9];               // dt * S22[q][q0 + t] - [t == q - q0] dtq: likewise for f2
  const double *F1new_p;          // coarse F at node p of the new sweep, NV comps
  const double *F1old[5];            // old coarse F at every coarse node
  const double *F2old[9];            // old fine F at the group's nodes, ns comps
  double *F2new[9];                  // new fine F at the group's nodes
  int eval_first;                 // evaluate f2 at node q0 (false only for q0 = 0)
  int eval_last;                  // evaluate f2 at node q0 + nsub after the last substep
};
void launch_fine_chain(const DevState &s, const double *U0, double *U, const FineChain &fc,
                       cudaStream_t st);
void launch_chem_only(const DevState &s, const double *U, double *F2, cudaStream_t st);
void launch_exp(const Mech *m, const double *x, double *y, long long n, int variant,
                cudaStream_t st);
void launch_dmul(const double *a, const double *b, double *y, long long n, cudaStream_t st);

// Implicit reaction integration over one coarse interval (MRSDC mode 2,
// kernels_bdf.cu): per cell, dU/dtau = R(U) + G on [0, dtp] by the BDF
// method.  Rbar (ns comps, nullable) receives (y(dtp) - y(0)) / dtp - G_Y,
// Uout (nv comps, nullable) the state at dtp.
struct BdfParams {
  const double *U;                // [nv][ncells] state at tau = 0
  const double *G;                // [nv][ncells] constant forcing, or null (zero)
  const double *F0;               // [ns][ncells] R(U) at tau = 0 if known, or null
  double *Rbar;
  double *Uout;
  unsigned long long *counters;   // [5]: steps, rejected, Newton failures, evaluations,
                                  //   max steps of a cell (nullable)
  double dtp, rtol, atol, eta;    // interval, tolerances, Newton tolerance
  double gam[6];                  // gamma_k = sum_{j<=k} 1/j
  int max_attempts;
};
int bdf_species_limit();
void launch_react_bdf(const DevState &s, const BdfParams &P, cudaStream_t st);

// Weights and sources of the collocation residual (device-resident table).
constexpr int SMC_RES_MAX = 80;
struct ResidualTable {
  int n1, n2;
  double c1[SMC_RES_MAX], c2[SMC_RES_MAX];
  const double *src1[SMC_RES_MAX];
  const double *src2[SMC_RES_MAX];
};
void launch_residual(const double *U0, const double *UM, const ResidualTable *tab, int nv,
                     long long NI, unsigned long long *out, cudaStream_t st);

}  // namespace smc
