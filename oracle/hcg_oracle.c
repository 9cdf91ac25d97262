/*
 * hcg_oracle.c -- plain, slow, FP64 CPU oracle for HCGrid convolution gridding.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this file.  The product
 * path (the CUDA library) never links, calls or includes it, and this file
 * shares no code, header, constant or table with it.
 *
 * What it computes (HCGrid, Wang et al. 2020, MNRAS; arXiv 2012.13173):
 *   - Eq. (1), Sec. 2.1: V[g] = (1/W_g) sum_n V[s_n] w(g; s_n),
 *                        W_g  = sum_n w(g; s_n)
 *     over the samples inside the kernel support (Sec. 3.6 item 3: the
 *     "sphere_radius" is the kernel's range of influence).  Gaussian kernel,
 *     w = exp(-d^2 / (2 sigma^2)), d = great-circle distance (haversine).
 *   - Sec. 3.2 / Sec. 3.3 step I: HEALPix RING pixel index of every sample,
 *     using the ring-scheme formulas of Gorski et al. 2005 (ApJ 622, 759),
 *     restated here from the published equations.
 *   - Sec. 3.3 step I: key-value sort of (pixel, sample index) into
 *     non-descending order; Sec. 3.3 step II: first-level lookup table
 *     pixel -> S_start; Sec. 3.3 step III: second-level table ring -> R_start.
 *   - Sec. 3.4: the contributing-sample set of each cell, obtained here by
 *     brute force (every pair) or by a sorted-latitude band search; neither
 *     uses the HEALPix tables, so they pin the table-driven search.
 *
 * Readings of points the paper leaves open:
 *   - support is the closed disc h <= h_R in the haversine domain;
 *   - the plain grid is lon/lat ("CAR" in the API): cell (i, j) is centred at
 *     lon0 + (i - (nx-1)/2) * pix, lat0 + (j - (ny-1)/2) * pix (degrees);
 *     projected grids follow the FITS conventions (orc_wcs_cells);
 *   - longitude offsets are taken relative to lon0 and wrapped to (-180, 180];
 *   - ties in the pixel sort are broken by a 32-bit coordinate hash
 *     (MurmurHash3 fmix64 finaliser, Appleby) and then by sample index, so
 *     that the sorted order does not depend on the input order;
 *   - empty cells (W = 0) give V = NaN.
 *
 * Compile with -ffp-contract=off: every FP64 operation here is a separately
 * rounded IEEE operation, as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
static const double ORC_DEG = ORC_PI / 180.0;   /* degrees -> radians */

/* ------------------------------------------------------------------------ */
/* HEALPix RING scheme (Gorski et al. 2005, Sec. 4 and Eqs. 4-9).           */
/* Rings are numbered 1 .. 4*nside-1 from the north pole.  Ring r holds     */
/* 4r pixels for r < nside (north cap), 4*nside in the equatorial belt      */
/* nside <= r <= 3*nside, and 4*(4*nside - r) in the south cap.             */
/* ------------------------------------------------------------------------ */

int64_t orc_npix(int64_t nside) { return 12 * nside * nside; }

int64_t orc_ring_npix(int64_t nside, int64_t r)
{
    if (r < nside) return 4 * r;
    if (r > 3 * nside) return 4 * (4 * nside - r);
    return 4 * nside;
}

/* First pixel of ring r (also valid for r = 4*nside, giving npix). */
int64_t orc_ring_start(int64_t nside, int64_t r)
{
    if (r <= nside) return 2 * r * (r - 1);
    if (r <= 3 * nside) return 2 * nside * (nside - 1) + (r - nside) * 4 * nside;
    int64_t q = 4 * nside - r;                  /* rings left to the south pole */
    return orc_npix(nside) - 2 * q * (q + 1);
}

/* Ring number of a pixel, found by walking the ring starts (slow, plain). */
int64_t orc_pix2ring(int64_t nside, int64_t pix)
{
    int64_t lo = 1, hi = 4 * nside - 1;        /* largest r with start(r) <= pix */
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (orc_ring_start(nside, mid) <= pix) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* Longitude (degrees) reduced to [0, 360). */
static double orc_lon360(double lon)
{
    double l = fmod(lon, 360.0);
    if (l < 0.0) l = l + 360.0;
    if (l >= 360.0) l = 0.0;
    return l;
}

/*
 * ang2pix, RING scheme.  z = cos(theta) = sin(lat); phi = longitude.
 * t = phi / (pi/2) in [0, 4) is formed as lon/90 in degrees.
 * Equatorial belt (|z| <= 2/3): the two edge-line indices
 *   j+ = floor(nside (1/2 + t) - (3/4) nside z),  j- = floor(nside (1/2 + t) + (3/4) nside z)
 * give the ring (counted from z = 2/3) i = nside + 1 + j+ - j- and the index
 * in the ring (j+ + j- - nside + 1 + shift) / 2.
 * Polar caps (|z| > 2/3): with tp = frac(t) and x = nside sqrt(3 (1 - |z|)),
 *   j+ = floor(tp x), j- = floor((1 - tp) x), ring from the pole i = j+ + j- + 1,
 * index in the ring floor(t i).
 */
int64_t orc_ang2pix(int64_t nside, double lon_deg, double lat_deg, int64_t *ring_out)
{
    double z = sin(lat_deg * ORC_DEG);
    double za = fabs(z);
    double tt = orc_lon360(lon_deg) / 90.0;
    if (tt >= 4.0) tt = tt - 4.0;
    double ns = (double)nside;
    int64_t pix, ring;
    if (za <= 2.0 / 3.0) {
        double t1 = ns * (0.5 + tt);
        double t2 = (ns * 0.75) * z;
        int64_t jp = (int64_t)floor(t1 - t2);
        int64_t jm = (int64_t)floor(t1 + t2);
        int64_t ir = nside + 1 + jp - jm;       /* 1 .. 2 nside + 1 */
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - nside + kshift + 1) / 2;
        ip = ip % (4 * nside);
        pix = 2 * nside * (nside - 1) + (ir - 1) * 4 * nside + ip;
        ring = nside - 1 + ir;
    } else {
        double tp = tt - floor(tt);
        double x = ns * sqrt(3.0 * (1.0 - za));
        int64_t jp = (int64_t)floor(tp * x);
        int64_t jm = (int64_t)floor((1.0 - tp) * x);
        int64_t ir = jp + jm + 1;               /* 1 .. nside */
        int64_t ip = (int64_t)floor(tt * (double)ir);
        ip = ip % (4 * ir);
        if (z > 0.0) { pix = 2 * ir * (ir - 1) + ip; ring = ir; }
        else { pix = orc_npix(nside) - 2 * ir * (ir + 1) + ip; ring = 4 * nside - ir; }
    }
    if (ring_out) *ring_out = ring;
    return pix;
}

/* Centre of a RING pixel (Gorski et al. 2005, Eqs. 4-9), in degrees. */
void orc_pix2ang(int64_t nside, int64_t pix, double *lon_deg, double *lat_deg)
{
    int64_t r = orc_pix2ring(nside, pix);
    int64_t j = pix - orc_ring_start(nside, r);          /* 0-based in ring */
    double ns = (double)nside, z, phi;
    if (r < nside) {
        z = 1.0 - (double)(r * r) / (3.0 * ns * ns);
        phi = (ORC_PI / (2.0 * (double)r)) * ((double)j + 0.5);
    } else if (r <= 3 * nside) {
        z = 4.0 / 3.0 - 2.0 * (double)r / (3.0 * ns);
        int64_t s = (r - nside + 1) % 2;      /* 1 on rings shifted by half a pixel */
        phi = (ORC_PI / (2.0 * ns)) * ((double)j + 0.5 * (double)s);
    } else {
        int64_t q = 4 * nside - r;
        z = -1.0 + (double)(q * q) / (3.0 * ns * ns);
        phi = (ORC_PI / (2.0 * (double)q)) * ((double)j + 0.5);
    }
    *lat_deg = asin(z) / ORC_DEG;
    *lon_deg = phi / ORC_DEG;
}

/* ------------------------------------------------------------------------ */
/* Gridding geometry (Sec. 2.1, Eq. 1; Sec. 3.6 item 3).                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double lon0, lat0, pix;   /* grid centre and cell size, degrees */
    int64_t nx, ny;
    double R;                 /* support radius, degrees ("sphere_radius") */
    double fwhm;              /* Gaussian FWHM, degrees */
    const double *clon, *clat;   /* explicit cell centres [ny][nx] (degrees), or NULL: plain lon/lat grid */
} orc_geom;

static double orc_wrap180(double x)
{
    double y = fmod(x, 360.0);
    if (y > 180.0) y = y - 360.0;
    if (y <= -180.0) y = y + 360.0;
    return y;
}

/* sigma of the Gaussian kernel, radians: FWHM / (2 sqrt(2 ln 2)). */
static double orc_sigma(const orc_geom *g) { return (g->fwhm * ORC_DEG) / sqrt(8.0 * log(2.0)); }

/* h_R = sin^2(R/2): the support boundary in the haversine domain. */
double orc_hR(double R_deg)
{
    double s = sin(0.5 * (R_deg * ORC_DEG));
    return s * s;
}

/* Haversine of the great-circle distance between cell (i, j) and a sample. */
double orc_hav(const orc_geom *g, int64_t i, int64_t j, double lon, double lat)
{
    if (g->clon) {            /* explicit cell centre */
        double lonc = g->clon[j * g->nx + i], latc = g->clat[j * g->nx + i];
        double dlon = orc_wrap180(lon - lonc) * ORC_DEG;
        double dlat = (lat - latc) * ORC_DEG;
        double cg = cos(latc * ORC_DEG);
        double cn = cos(lat * ORC_DEG);
        double sd = sin(0.5 * dlat);
        double sa = sin(0.5 * dlon);
        return sd * sd + (cg * cn) * (sa * sa);
    }
    double a = ((double)i - 0.5 * (double)(g->nx - 1)) * g->pix;   /* cell lon - lon0 */
    double b = ((double)j - 0.5 * (double)(g->ny - 1)) * g->pix;   /* cell lat - lat0 */
    double dlon = (orc_wrap180(lon - g->lon0) - a) * ORC_DEG;
    double dlat = ((lat - g->lat0) - b) * ORC_DEG;
    double cg = cos((g->lat0 + b) * ORC_DEG);
    double cn = cos(lat * ORC_DEG);
    double sd = sin(0.5 * dlat);
    double sa = sin(0.5 * dlon);
    return sd * sd + (cg * cn) * (sa * sa);
}

/* Kernel weight from the haversine value: d = 2 asin(sqrt h). */
double orc_weight(const orc_geom *g, double h)
{
    double d = 2.0 * asin(sqrt(h));
    double s = orc_sigma(g);
    return exp(-(d * d) / (2.0 * s * s));
}

static void orc_fill_geom(orc_geom *g, const double *p)
{
    g->lon0 = p[0]; g->lat0 = p[1]; g->pix = p[2];
    g->nx = (int64_t)p[3]; g->ny = (int64_t)p[4];
    g->R = p[5]; g->fwhm = p[6];
    g->clon = NULL; g->clat = NULL;
}

/* ------------------------------------------------------------------------ */
/* Grid projections (Calabretta & Greisen 2002, the FITS world coordinate   */
/* conventions the paper's WCS grids follow, Sec. 2.1).                      */
/* ------------------------------------------------------------------------ */
/*
 * Cell (i, j) has offsets x = (i - (nx-1)/2) pix eastward and
 * y = (j - (ny-1)/2) pix northward (degrees) from the reference point
 * (lon0, lat0) at the grid centre.  With r0 the unit vector of the reference
 * point and e0, n0 the local east and north unit vectors there:
 *   proj 1 TAN: distance rho = atan(|(x, y)|), bearing b = atan2(x, y) east of
 *               north: v = cos rho r0 + sin rho (cos b n0 + sin b e0)
 *   proj 2 SIN: the same with rho = asin(|(x, y)|) (|(x, y)| <= 1 rad)
 *   proj 3 SFL: native (phi, theta) = (x / cos y, y),
 *   proj 4 CAR: native (phi, theta) = (x, y); for both
 *               v = cos theta cos phi r0 + cos theta sin phi e0 + sin theta n0,
 *               the native equator being the great circle through the
 *               reference point heading east (plain lon/lat when lat0 = 0).
 * Writes the cell centres (lon in [0, 360), lat) in degrees; returns the
 * number of cells a projection cannot place (NaN written there).
 */
int64_t orc_wcs_cells(int proj, double lon0, double lat0, double pix, int64_t nx, int64_t ny,
                      double *clon, double *clat)
{
    double a0 = lon0 * ORC_DEG, d0 = lat0 * ORC_DEG;
    double r0[3] = {cos(d0) * cos(a0), cos(d0) * sin(a0), sin(d0)};
    double e0[3] = {-sin(a0), cos(a0), 0.0};
    double n0[3] = {-sin(d0) * cos(a0), -sin(d0) * sin(a0), cos(d0)};
    int64_t bad = 0;
    for (int64_t j = 0; j < ny; j++) {
        for (int64_t i = 0; i < nx; i++) {
            double x = ((double)i - 0.5 * (double)(nx - 1)) * pix * ORC_DEG;
            double y = ((double)j - 0.5 * (double)(ny - 1)) * pix * ORC_DEG;
            double cr, cn, ce;        /* components along r0, n0, e0 */
            int ok = 1;
            if (proj == 1 || proj == 2) {
                double R = sqrt(x * x + y * y);
                double rho;
                if (proj == 1) rho = atan(R);
                else { if (R > 1.0) ok = 0; rho = ok ? asin(R) : 0.0; }
                double b = atan2(x, y);
                cr = cos(rho); cn = sin(rho) * cos(b); ce = sin(rho) * sin(b);
            } else if (proj == 3 || proj == 4) {
                double th = y;
                double ph = x;
                if (proj == 3) { if (cos(th) <= 0.0) ok = 0; else ph = x / cos(th); }
                cr = cos(th) * cos(ph); ce = cos(th) * sin(ph); cn = sin(th);
            } else {
                ok = 0; cr = cn = ce = 0.0;
            }
            int64_t c = j * nx + i;
            if (!ok) { clon[c] = NAN; clat[c] = NAN; bad++; continue; }
            double v[3];
            for (int k = 0; k < 3; k++) v[k] = cr * r0[k] + cn * n0[k] + ce * e0[k];
            double lon = atan2(v[1], v[0]) / ORC_DEG;
            if (lon < 0.0) lon += 360.0;
            if (lon >= 360.0) lon = 0.0;
            double z = v[2] > 1.0 ? 1.0 : (v[2] < -1.0 ? -1.0 : v[2]);
            clon[c] = lon;
            clat[c] = asin(z) / ORC_DEG;
        }
    }
    return bad;
}

/*
 * Neighbour search by brute force: every (cell, sample) pair.
 * geom = {lon0, lat0, pix, nx, ny, R, fwhm}.
 * Writes counts[cells] (cells = nx*ny, row-major j*nx + i); if ids != NULL
 * also fills CSR ids using offsets[] (exclusive prefix of counts, supplied).
 * guard[cells] (optional) counts pairs with |h - h_R| <= gtol * h_R.
 */
void orc_neigh_brute_xy(const double *geom, const double *clon, const double *clat, int64_t n, const double *lon,
                        const double *lat, int64_t *counts, const int64_t *offsets, int64_t *ids, int64_t *guard,
                        double gtol);

void orc_neigh_brute(const double *geom, int64_t n, const double *lon, const double *lat,
                     int64_t *counts, const int64_t *offsets, int64_t *ids,
                     int64_t *guard, double gtol)
{
    orc_neigh_brute_xy(geom, NULL, NULL, n, lon, lat, counts, offsets, ids, guard, gtol);
}

/* Brute force with explicit cell centres clon/clat [ny][nx] (NULL: plain lon/lat grid). */
void orc_neigh_brute_xy(const double *geom, const double *clon, const double *clat, int64_t n, const double *lon,
                        const double *lat, int64_t *counts, const int64_t *offsets, int64_t *ids, int64_t *guard,
                        double gtol)
{
    orc_geom g; orc_fill_geom(&g, geom);
    g.clon = clon; g.clat = clat;
    double hR = orc_hR(g.R);
    int64_t cells = g.nx * g.ny;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < cells; c++) {
        int64_t i = c % g.nx, j = c / g.nx, k = 0, gk = 0;
        for (int64_t s = 0; s < n; s++) {
            double h = orc_hav(&g, i, j, lon[s], lat[s]);
            if (fabs(h - hR) <= gtol * hR) gk++;
            if (h <= hR) {
                if (ids) ids[offsets[c] + k] = s;
                k++;
            }
        }
        counts[c] = k;
        if (guard) guard[c] = gk;
    }
}

/* Sorted-latitude band search: a plain index of samples ordered by latitude. */
typedef struct { double lat; int64_t idx; } orc_latidx;

static int orc_cmp_lat(const void *a, const void *b)
{
    const orc_latidx *x = (const orc_latidx *)a, *y = (const orc_latidx *)b;
    if (x->lat < y->lat) return -1;
    if (x->lat > y->lat) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

static orc_latidx *orc_build_latidx(int64_t n, const double *lat)
{
    orc_latidx *t = (orc_latidx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_latidx));
    for (int64_t s = 0; s < n; s++) { t[s].lat = lat[s]; t[s].idx = s; }
    qsort(t, (size_t)n, sizeof(orc_latidx), orc_cmp_lat);
    return t;
}

/* first position with lat >= x */
static int64_t orc_lat_lower(const orc_latidx *t, int64_t n, double x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) { int64_t m = (lo + hi) / 2; if (t[m].lat < x) lo = m + 1; else hi = m; }
    return lo;
}

/* Contributors of one cell via the latitude band [lat_g - R - eps, lat_g + R + eps];
 * the ids are returned in increasing sample order. */
static int64_t orc_cell_band(const orc_geom *g, const orc_latidx *t, int64_t n,
                             const double *lon, const double *lat, int64_t i, int64_t j,
                             double hR, int64_t *ids, int64_t *guard, double gtol)
{
    double b = ((double)j - 0.5 * (double)(g->ny - 1)) * g->pix;
    double latg = g->clat ? g->clat[j * g->nx + i] : g->lat0 + b;
    double margin = g->R * (1.0 + 1e-9) + 1e-9;
    int64_t a0 = orc_lat_lower(t, n, latg - margin);
    int64_t a1 = orc_lat_lower(t, n, latg + margin);
    int64_t k = 0, gk = 0;
    for (int64_t q = a0; q < a1; q++) {
        int64_t s = t[q].idx;
        double h = orc_hav(g, i, j, lon[s], lat[s]);
        if (fabs(h - hR) <= gtol * hR) gk++;
        if (h <= hR) { if (ids) ids[k] = s; k++; }
    }
    if (guard) *guard = gk;
    return k;
}

static int orc_cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Band-search neighbour lists for a list of cells (cell index = j*nx + i).
 * Pass ids == NULL to get the counts only. */
void orc_neigh_band_xy(const double *geom, const double *clon, const double *clat, int64_t n, const double *lon,
                       const double *lat, int64_t ncell, const int64_t *cell, int64_t *counts,
                       const int64_t *offsets, int64_t *ids, int64_t *guard, double gtol);

void orc_neigh_band(const double *geom, int64_t n, const double *lon, const double *lat,
                    int64_t ncell, const int64_t *cell, int64_t *counts,
                    const int64_t *offsets, int64_t *ids, int64_t *guard, double gtol)
{
    orc_neigh_band_xy(geom, NULL, NULL, n, lon, lat, ncell, cell, counts, offsets, ids, guard, gtol);
}

/* The band search with explicit cell centres clon/clat [ny][nx] (NULL: plain lon/lat grid). */
void orc_neigh_band_xy(const double *geom, const double *clon, const double *clat, int64_t n, const double *lon,
                       const double *lat, int64_t ncell, const int64_t *cell, int64_t *counts,
                       const int64_t *offsets, int64_t *ids, int64_t *guard, double gtol)
{
    orc_geom g; orc_fill_geom(&g, geom);
    g.clon = clon; g.clat = clat;
    double hR = orc_hR(g.R);
    orc_latidx *t = orc_build_latidx(n, lat);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < ncell; q++) {
        int64_t c = cell[q], i = c % g.nx, j = c / g.nx, gk = 0;
        int64_t *dst = ids ? ids + offsets[q] : NULL;
        counts[q] = orc_cell_band(&g, t, n, lon, lat, i, j, hR, dst, &gk, gtol);
        if (dst) qsort(dst, (size_t)counts[q], sizeof(int64_t), orc_cmp_i64);
        if (guard) guard[q] = gk;
    }
    free(t);
}

/*
 * Eq. (1) for a list of cells, FP64 throughout.
 * spec: [n][nchan] row-major doubles.  out_v: [ncell][nchan], out_w: [ncell],
 * out_abs: [ncell][nchan] = sum_n w |s_n| / W (the scale used by the
 * condition-aware tolerance), out_cnt: contributors per cell.
 * W = 0 gives V = NaN and abs = 0.
 */
void orc_grid_cells_xy(const double *geom, const double *clon, const double *clat, int64_t n, const double *lon,
                       const double *lat, const double *spec, int64_t nchan, int64_t ncell, const int64_t *cell,
                       double *out_v, double *out_w, double *out_abs, int64_t *out_cnt);

void orc_grid_cells(const double *geom, int64_t n, const double *lon, const double *lat,
                    const double *spec, int64_t nchan, int64_t ncell, const int64_t *cell,
                    double *out_v, double *out_w, double *out_abs, int64_t *out_cnt)
{
    orc_grid_cells_xy(geom, NULL, NULL, n, lon, lat, spec, nchan, ncell, cell, out_v, out_w, out_abs, out_cnt);
}

/* Eq. (1) with explicit cell centres clon/clat [ny][nx] (NULL: plain lon/lat grid). */
void orc_grid_cells_xy(const double *geom, const double *clon, const double *clat, int64_t n, const double *lon,
                       const double *lat, const double *spec, int64_t nchan, int64_t ncell, const int64_t *cell,
                       double *out_v, double *out_w, double *out_abs, int64_t *out_cnt)
{
    orc_geom g; orc_fill_geom(&g, geom);
    g.clon = clon; g.clat = clat;
    double hR = orc_hR(g.R);
    orc_latidx *t = orc_build_latidx(n, lat);
#pragma omp parallel
    {
        int64_t *ids = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        double *acc = (double *)malloc((size_t)nchan * sizeof(double));
        double *aab = (double *)malloc((size_t)nchan * sizeof(double));
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < ncell; q++) {
            int64_t c = cell[q], i = c % g.nx, j = c / g.nx;
            int64_t k = orc_cell_band(&g, t, n, lon, lat, i, j, hR, ids, NULL, 0.0);
            qsort(ids, (size_t)k, sizeof(int64_t), orc_cmp_i64);
            double W = 0.0;
            for (int64_t ch = 0; ch < nchan; ch++) { acc[ch] = 0.0; aab[ch] = 0.0; }
            for (int64_t m = 0; m < k; m++) {
                int64_t s = ids[m];
                double w = orc_weight(&g, orc_hav(&g, i, j, lon[s], lat[s]));
                W += w;
                const double *row = spec + s * nchan;
                for (int64_t ch = 0; ch < nchan; ch++) {
                    acc[ch] += w * row[ch];
                    aab[ch] += w * fabs(row[ch]);
                }
            }
            out_w[q] = W;
            if (out_cnt) out_cnt[q] = k;
            for (int64_t ch = 0; ch < nchan; ch++) {
                out_v[q * nchan + ch] = (W > 0.0) ? acc[ch] / W : NAN;
                if (out_abs) out_abs[q * nchan + ch] = (W > 0.0) ? aab[ch] / W : 0.0;
            }
        }
        free(ids); free(acc); free(aab);
    }
    free(t);
}

/* ------------------------------------------------------------------------ */
/* Pre-ordering and the two-level lookup table (Sec. 3.3 steps I-III).      */
/* ------------------------------------------------------------------------ */

/* MurmurHash3 64-bit finaliser (fmix64, Appleby), restated. */
static uint64_t orc_fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* 32-bit tie-break hash of a sample's coordinates (raw IEEE bit patterns). */
uint32_t orc_coord_hash(double lon, double lat)
{
    uint64_t a, b;
    memcpy(&a, &lat, 8);
    memcpy(&b, &lon, 8);
    uint64_t x = a ^ ((b << 29) | (b >> 35));
    return (uint32_t)(orc_fmix64(x) >> 32);
}

typedef struct { int64_t pix; uint32_t hash; int64_t idx; } orc_sortrec;

static int orc_cmp_rec(const void *a, const void *b)
{
    const orc_sortrec *x = (const orc_sortrec *)a, *y = (const orc_sortrec *)b;
    if (x->pix != y->pix) return (x->pix < y->pix) ? -1 : 1;
    if (x->hash != y->hash) return (x->hash < y->hash) ? -1 : 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/*
 * Step I: pixel index of every sample; keep the samples whose ring lies in
 * [r_lo, r_hi] (the rings the grid can reach) and sort them by
 * (pixel, coordinate hash, sample index).  Writes the sorted pixels P' and
 * sample indices (the permutation giving S'), returns M (samples kept).
 */
int64_t orc_preorder(int64_t nside, int64_t n, const double *lon, const double *lat,
                     int64_t r_lo, int64_t r_hi, int64_t *pix_sorted, int64_t *perm)
{
    orc_sortrec *t = (orc_sortrec *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_sortrec));
    int64_t m = 0;
    for (int64_t s = 0; s < n; s++) {
        int64_t ring;
        int64_t p = orc_ang2pix(nside, lon[s], lat[s], &ring);
        if (ring < r_lo || ring > r_hi) continue;
        t[m].pix = p; t[m].hash = orc_coord_hash(lon[s], lat[s]); t[m].idx = s;
        m++;
    }
    qsort(t, (size_t)m, sizeof(orc_sortrec), orc_cmp_rec);
    for (int64_t q = 0; q < m; q++) { pix_sorted[q] = t[q].pix; perm[q] = t[q].idx; }
    free(t);
    return m;
}

/* Step II: first-level table.  upix[k] = k-th distinct pixel of P',
 * ustart[k] = smallest index q with P'[q] == upix[k]; ustart[U] = M.  Returns U. */
int64_t orc_lut1(int64_t m, const int64_t *pix_sorted, int64_t *upix, int64_t *ustart)
{
    int64_t u = 0;
    for (int64_t q = 0; q < m; q++) {
        if (q == 0 || pix_sorted[q] != pix_sorted[q - 1]) { upix[u] = pix_sorted[q]; ustart[u] = q; u++; }
    }
    ustart[u] = m;
    return u;
}

/* Step III: second-level table.  For r in [r_lo, r_hi + 1]:
 * rstart[r - r_lo] = smallest index q with ring(P'[q]) >= r (M if none). */
void orc_lut2(int64_t nside, int64_t m, const int64_t *pix_sorted, int64_t r_lo, int64_t r_hi,
              int64_t *rstart)
{
    int64_t q = 0;   /* ring(P'[q]) is non-decreasing, so the scan never restarts */
    for (int64_t r = r_lo; r <= r_hi + 1; r++) {
        while (q < m && orc_pix2ring(nside, pix_sorted[q]) < r) q++;
        rstart[r - r_lo] = q;
    }
}

/* ------------------------------------------------------------------------ */
/* Kernel parameter rules (Sec. 3.6 item 3).                                 */
/* ------------------------------------------------------------------------ */

/* Smallest power-of-two nside whose mean pixel size sqrt(pi/3)/nside is at
 * most sigma_kernel / 2 ("hpx_max_resolution ~ sigma_kernel/2"). */
int64_t orc_nside_for(double fwhm_deg)
{
    double sig = (fwhm_deg * ORC_DEG) / sqrt(8.0 * log(2.0));
    int64_t ns = 1;
    while (sqrt(ORC_PI / 3.0) / (double)ns > 0.5 * sig && ns < ((int64_t)1 << 29)) ns *= 2;
    return ns;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
