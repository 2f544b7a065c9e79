// Host-only geometry helpers (host_geom.cu).
#pragma once
#include <functional>
#include <vector>

#include "ffe_internal.h"
#include "shellmap.cuh"

namespace ffe {

// x(xi) and d xi / d x of element e
typedef std::function<void(int e, const double xi[3], double x[3], double ijac[3][3])> MapFn;

void ks_point(const double x[3], double M, double a, double out[NMET]);
void wald_point(const double x[3], double M, double a, double B0, double U[NV]);
void dipole_point(const double x[3], double mu, double delta, double chi, double U[NV]);
void match_faces(int E, const MapFn& map, const std::vector<double>& xnodes, int np1, double scale,
                 std::vector<int>& nbr, std::vector<int>& nbf, std::vector<int>& orient);
// Reference coordinates xn, in element eln of shell geometry gn, of the centre of
// ghost cell (g, ta, tb) past face (dd, s) of element el of geometry ge (the
// element's reference grid continued past the face, mapped by its wedge map,
// taken back by the neighbour's closed-form inverse map).
void shell_ghost_ref(const ShellGeo& ge, int el, const ShellGeo& gn, int eln, int dd, int s, int g, int ta, int tb,
                     int nc, double xn[3]);
// 6-point Lagrange weights w[6] at t through the 6 subcell centres nearest t
// (stencil kept inside the nc cells); returns its first cell.
int fd6_stencil(int nc, double t, double* w);
// Lagrange weights w[n] at t through the nodes x[0..n).
void lagrange_at(const double* x, int n, double t, double* w);

}  // namespace ffe
