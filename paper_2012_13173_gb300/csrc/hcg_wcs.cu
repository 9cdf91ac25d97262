// hcg_wcs.cu -- cell centres of projected target grids (host code).
//
// The FITS world-coordinate conventions (Calabretta & Greisen 2002) for the
// projections hcg_set_grid offers, with the reference pixel at the grid
// centre (CRPIX), CDELT = (+pixel, +pixel) and the default native longitude
// of the celestial pole.  A cell's intermediate coordinates (x, y) give its
// native direction u in a frame whose first axis points at the reference
// point, second axis east and third axis north there:
//   TAN / SIN   zenithal: native distance rho = atan(r) / asin(r) from the
//               reference point, r = |(x, y)| in radians, at bearing
//               beta = atan2(x, y) east of north:
//               u = (cos rho, sin rho sin beta, sin rho cos beta)
//   CAR / SFL   cylindrical / pseudo-cylindrical: native (phi, theta) =
//               (x, y) / (x / cos y, y):
//               u = (cos theta cos phi, cos theta sin phi, sin theta)
// and the celestial direction is v = Rz(lon0) Ry(-lat0) u.
#include <math.h>

#include "hcg_internal.h"

namespace {

constexpr double kRad = 3.14159265358979323846 / 180.0;

// v = Rz(a) Ry(-d) u: the rotation taking (1, 0, 0) to the reference point
// (a, d), (0, 1, 0) to its local east and (0, 0, 1) to its local north.
void to_celestial(double a, double d, const double u[3], double v[3]) {
    const double cd = cos(d), sd = sin(d), ca = cos(a), sa = sin(a);
    const double w0 = cd * u[0] - sd * u[2];       // Ry(-d)
    const double w2 = sd * u[0] + cd * u[2];
    v[0] = ca * w0 - sa * u[1];                    // Rz(a)
    v[1] = sa * w0 + ca * u[1];
    v[2] = w2;
}

}  // namespace

// Cell centres (degrees; lon in [0, 360)) of an nx x ny grid in projection
// proj; returns the number of cells the projection cannot place (SIN beyond
// its hemisphere, SFL or CAR at |y| >= 90 degrees), whose entries are NaN.
int wcs_cell_centres(int proj, double lon0, double lat0, double pix, int nx, int ny, double *lon, double *lat) {
    const double a0 = lon0 * kRad, d0 = lat0 * kRad;
    int bad = 0;
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            const double x = (i - 0.5 * (nx - 1)) * pix * kRad, y = (j - 0.5 * (ny - 1)) * pix * kRad;
            double u[3];
            bool ok = true;
            if (proj == HCG_WCS_TAN || proj == HCG_WCS_SIN) {
                const double r = hypot(x, y);
                if (proj == HCG_WCS_SIN && r > 1.0) ok = false;
                const double rho = proj == HCG_WCS_TAN ? atan(r) : (ok ? asin(r) : 0.0);
                const double beta = atan2(x, y);
                u[0] = cos(rho); u[1] = sin(rho) * sin(beta); u[2] = sin(rho) * cos(beta);
            } else {
                const double theta = y;
                double phi = x;
                if (fabs(theta) >= 0.5 * 3.14159265358979323846) ok = false;
                else if (proj == HCG_WCS_SFL) phi = x / cos(theta);
                u[0] = cos(theta) * cos(phi); u[1] = cos(theta) * sin(phi); u[2] = sin(theta);
            }
            const size_t k = (size_t)j * nx + i;
            if (!ok) { lon[k] = NAN; lat[k] = NAN; bad++; continue; }
            double v[3];
            to_celestial(a0, d0, u, v);
            double l = atan2(v[1], v[0]) / kRad;
            if (l < 0.0) l += 360.0;
            if (l >= 360.0) l -= 360.0;
            lon[k] = l;
            lat[k] = asin(fmax(-1.0, fmin(1.0, v[2]))) / kRad;
        }
    }
    return bad;
}
