// em.cu -- transverse fields of the co-rotating frame (App. A) in the 1D
// reduction: every quantity depends on h alone, B = B_* h-hat + B_perp, and
// the frame moves at beta = (0, beta_y, beta_z) across h.  In code units
// (c = 1, 4 pi absorbed; d = d/dh) App. A's Maxwell equations read
//   dB_y/dt = d E_z,          dB_z/dt = -d E_y,
//   dE_y/dt = -d B_z + jv_y,  dE_z/dt = d B_y + jv_z,
// and jv_h joins the Ampere step of E_h; with P = beta (beta . B) - |beta|^2 B_perp
// the virtual current -{curl(beta x E) + beta x curl E - curl[beta x (beta x B)]}
// has the components
//   jv_h = -(beta_y d E_y + beta_z d E_z),
//   jv_y = -beta_y d E_h - d P_z,   jv_z = -beta_z d E_h + d P_y.
// Particles move along B_* (the strong-field limit); with jperp their guiding
// centres' transverse current j_perp (deposited by the push kernels in em_jy,
// em_jz) joins the cells' update, dE_perp/dt = ... - j_perp, and is cleared
// here for the next step.
//
// Yee grid, second order: E_y, E_z on cell centres at half steps; B_y, B_z
// on nodes at whole steps.  Both kernels run after the push and before the
// deferred Ampere step, while E[e_cur] still holds E_h^n:
//   k_em_cells  E_perp^{n-1/2} -> E_perp^{n+1/2} from B^n and d E_h^n
//   k_em_nodes  B^n -> B^{n+1} from d E_perp^{n+1/2}; Jv = dt jv_h^{n+1/2}
//               for the Ampere step (filter.cu adds it unsmoothed)
// Surface gap: conductors at the star (node 0) and at the top (node nx):
// a cell beyond either end is the image of the cell inside with its sign
// reversed (E_perp = 0 on a conductor).  Below the top an absorbing layer of
// pml_cells cells: matched electric and magnetic conductivity
// sigma(X) = pml_smax ((X - X_p)/pml_cells)^3 above X_p = nx - pml_cells
// (Berenger's layer, which in 1D needs no field splitting); every field is
// advanced as F <- a F + b (rhs), a = (1 - sigma dt/2)/(1 + sigma dt/2),
// b = dt/(1 + sigma dt/2).  Periodic gap: both grids wrap.
//
// One block per tile; each kernel writes only its own tile's entries and
// reads the neighbours' entries of arrays it does not write, so the two
// launches need no other ordering.  Each node costs a few doubles of
// traffic; the kernels are field-only and small next to the push.
#include "gap_internal.cuh"
#include "kernels.h"

namespace gapk {

__device__ __forceinline__ double layer_sigma(const GapDev &g, double X) {
  if (g.periodic || g.pml_cells <= 0) return 0.0;
  const double Xp = (double)(g.nx - g.pml_cells);
  if (!(X > Xp)) return 0.0;
  const double f = (X - Xp) / (double)g.pml_cells;
  return g.pml_smax * f * f * f;
}

__global__ void __launch_bounds__(256) k_em_cells(View v) {
  const TileDev ti = v.tiles[blockIdx.x];
  const GapDev &g = v.gaps[ti.gap];
  if (!g.em) return;
  const double *E = v.E[v.ctl->e_cur] + g.node_off;
  const double *By = v.em_By + g.node_off, *Bz = v.em_Bz + g.node_off;
  double *Ey = v.em_Ey + g.node_off, *Ez = v.em_Ez + g.node_off;
  const double by = g.beta_y, bz = g.beta_z, b2 = by * by + bz * bz, dx = g.dx, dt = g.dt;
  for (int k = threadIdx.x; k < ti.nk; k += blockDim.x) {
    const int64_t c = (int64_t)ti.k0 + k;
    if (c >= g.nx) continue;  // the top node of a surface gap has no cell
    const int64_t i0 = c, i1 = g.periodic && c + 1 == g.nx ? 0 : c + 1;
    const double dEh = (E[i1] - E[i0]) / dx;
    const double By0 = By[i0], By1 = By[i1], Bz0 = Bz[i0], Bz1 = Bz[i1];
    const double bB0 = by * By0 + bz * Bz0, bB1 = by * By1 + bz * Bz1;
    const double Py0 = by * bB0 - b2 * By0, Py1 = by * bB1 - b2 * By1;
    const double Pz0 = bz * bB0 - b2 * Bz0, Pz1 = bz * bB1 - b2 * Bz1;
    const double jvy = -by * dEh - (Pz1 - Pz0) / dx;
    const double jvz = -bz * dEh + (Py1 - Py0) / dx;
    double ry = -(Bz1 - Bz0) / dx + jvy;
    double rz = (By1 - By0) / dx + jvz;
    if (g.jperp) {
      double *jy = v.em_jy + g.node_off, *jz = v.em_jz + g.node_off;
      ry -= jy[c];
      rz -= jz[c];
      jy[c] = 0.0;
      jz[c] = 0.0;
    }
    const double sg = layer_sigma(g, (double)c + 0.5);
    const double a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt), b = dt / (1.0 + 0.5 * sg * dt);
    Ey[c] = a * Ey[c] + b * ry;
    Ez[c] = a * Ez[c] + b * rz;
  }
}

__global__ void __launch_bounds__(256) k_em_nodes(View v) {
  const TileDev ti = v.tiles[blockIdx.x];
  const GapDev &g = v.gaps[ti.gap];
  if (!g.em) return;
  const double *Ey = v.em_Ey + g.node_off, *Ez = v.em_Ez + g.node_off;
  double *By = v.em_By + g.node_off, *Bz = v.em_Bz + g.node_off, *Jv = v.em_Jv + g.node_off;
  const double by = g.beta_y, bz = g.beta_z, dx = g.dx, dt = g.dt;
  for (int k = threadIdx.x; k < ti.nk; k += blockDim.x) {
    const int64_t i = (int64_t)ti.k0 + k;
    const double dEy = (cell_at(Ey, i, g) - cell_at(Ey, i - 1, g)) / dx;
    const double dEz = (cell_at(Ez, i, g) - cell_at(Ez, i - 1, g)) / dx;
    const double sg = layer_sigma(g, (double)i);
    const double a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt), b = dt / (1.0 + 0.5 * sg * dt);
    Bz[i] = a * Bz[i] - b * dEy;
    By[i] = a * By[i] + b * dEz;
    Jv[i] = -dt * (by * dEy + bz * dEz);
  }
}

void launch_em(const View &v, cudaStream_t st) {
  if (!v.em_any) return;
  k_em_cells<<<v.n_tiles, 256, 0, st>>>(v);
  k_em_nodes<<<v.n_tiles, 256, 0, st>>>(v);
}

}  // namespace gapk
