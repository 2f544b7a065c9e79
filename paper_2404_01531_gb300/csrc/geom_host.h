// Host-only geometry helpers (host_geom.cu).
#pragma once
#include <functional>
#include <vector>

#include "ffe_internal.h"

namespace ffe {

// x(xi) and d xi / d x of element e
typedef std::function<void(int e, const double xi[3], double x[3], double ijac[3][3])> MapFn;

void ks_point(const double x[3], double M, double a, double out[NMET]);
void wald_point(const double x[3], double M, double a, double B0, double U[NV]);
void dipole_point(const double x[3], double mu, double delta, double chi, double U[NV]);
void match_faces(int E, const MapFn& map, const std::vector<double>& xnodes, int np1, double scale,
                 std::vector<int>& nbr, std::vector<int>& nbf, std::vector<int>& orient);

}  // namespace ffe
