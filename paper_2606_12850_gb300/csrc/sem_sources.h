// Host-side placement of sources between GLL nodes (libsemgb): point location in trilinear
// hexahedra and the Lagrange interpolation of point forces and moment tensors. Float64,
// deterministic; used by sem_capi.cpp.
#pragma once

#include <cstdint>

namespace semgb {

// Lagrange basis of the ngll nodes xi at an arbitrary x in [-1, 1]: l[i] = l_i(x) and
// dl[i] = l_i'(x). hprime[i*ngll + l] = l_l'(xi_i) is the nodal derivative matrix.
void lagrange_at(int ngll, const double* xi, const double* hprime, double x, double* l, double* dl);

// Lowest-numbered element of ctrl[nspec][8][3] that holds the point x[3], and its reference
// coordinates ref[3] in [-1, 1]; -1 if no element holds it.
int locate_point(int nspec, const double* ctrl, const double* x, double* ref);

// The same for npts points xyz[npts][3] (elem[npts], ref[npts][3]); for more than a few
// points the candidate elements come from a uniform grid of buckets over the elements'
// bounding boxes, with identical results.
void locate_points(int nspec, const double* ctrl, int npts, const double* xyz, int32_t* elem, double* ref);

// Nodal forces f[ngll^3][3] (local point order) of a point source at reference
// coordinates ref[3] of the element with corners ctrl_e[8][3]: force[3] gives
// f_p = F psi_p, moment[6] = (Mxx, Myy, Mzz, Mxy, Mxz, Myz) gives f_p = M grad psi_p;
// exactly one of them is non-NULL.
void point_source_forces(int ngll, const double* xi, const double* hprime, const double* ctrl_e,
                         const double* ref, const double* force, const double* moment, double* f);

}  // namespace semgb
