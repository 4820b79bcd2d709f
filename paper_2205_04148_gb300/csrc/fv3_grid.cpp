// fv3_grid.cpp -- host-side grid construction and halo plans (FP64).
//
// Grid (paper Section II: "gnomonic cubed-sphere grid"): equiangular gnomonic
// projection of each of the six cube faces; tile t maps scaled angles
// (sa, sb) in [-1, 1] to normalise(c + tan(sa pi/4) a + tan(sb pi/4) b) with
// the tile frames of the C-ABI (include/fv3.h).  Metric terms: great-circle
// edge and centre-to-centre lengths, spherical-excess cell and dual-cell
// areas, the cosine/sine of the angle between the two coordinate lines at each
// face, Coriolis 2*Omega*z at cells and corners.  A doubly-periodic uniform
// tile is the flat special case.
//
// Halo plans (Section V-C: halo updates must transform data according to the
// orientation of the adjoining cube faces; Section V-B: corner and edge
// specialisations): every halo slot of every tile is resolved, once, to the
// tile, position and sign of the value it must hold.  A strip slot is the
// neighbour's own cell or face, reached by the map that identifies the shared
// edge; tile-edge faces stored by two tiles take the value of the tile with
// the lower index; the three cells missing at a cube corner are read as the
// adjacent strip turned by 90 degrees about the corner (x-sweeps from the W/E
// strip, y-sweeps from the S/N strip).  Vector components move with the
// signed permutation of the two index bases.
#include "fv3_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace fv3 {

namespace {

struct V3 {
  double x, y, z;
};
inline V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 scale(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double len(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return scale(a, 1.0 / len(a)); }

// cube frames of the C-ABI convention: centre, alpha axis, beta axis
const int kTileFrame[6][3][3] = {
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},  {{0, 1, 0}, {-1, 0, 0}, {0, 0, 1}},
    {{-1, 0, 0}, {0, -1, 0}, {0, 0, 1}}, {{0, -1, 0}, {1, 0, 0}, {0, 0, 1}},
    {{0, 0, 1}, {0, 1, 0}, {-1, 0, 0}},  {{0, 0, -1}, {0, 1, 0}, {1, 0, 0}}};

V3 frame_vec(int t, int r) {
  return {double(kTileFrame[t][r][0]), double(kTileFrame[t][r][1]), double(kTileFrame[t][r][2])};
}

double tan_quarter(double s) {  // tan(s*pi/4), exactly +-1 on the tile edges
  if (s >= 1.0) return 1.0;
  if (s <= -1.0) return -1.0;
  return std::tan(s * 0.78539816339744830962);
}

// 2x2 signed permutation acting on index displacements; col c = image of e_c
struct Rot {
  int m[2][2] = {{1, 0}, {0, 1}};  // m[row][col]
  void image(int c, int& ax, int& ay) const { ax = m[0][c]; ay = m[1][c]; }
};
Rot compose(const Rot& after, const Rot& before) {  // after * before
  Rot r;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) r.m[a][b] = after.m[a][0] * before.m[0][b] + after.m[a][1] * before.m[1][b];
  return r;
}

// the four tile sides as frames in index space (units of n for the origin)
struct Side {
  int ox, oy;    // origin / n
  int tx, ty;    // unit along the side (increasing index)
  int nx, ny;    // unit outward normal
};
const Side kSide[4] = {{0, 0, 0, 1, -1, 0}, {1, 0, 0, 1, 1, 0}, {0, 0, 1, 0, 0, -1}, {0, 1, 1, 0, 0, 1}};

}  // namespace

// ---------------------------------------------------------------------------
struct Topology {
  int n = 0;
  bool cubed = false;
  int nbr_tile[6][4], nbr_side[6][4];
  bool nbr_flip[6][4];

  V3 point(int t, double X, double Y) const {
    double sa = (2.0 * X - n) / n, sb = (2.0 * Y - n) / n;
    V3 p = add(frame_vec(t, 0), add(scale(frame_vec(t, 1), tan_quarter(sa)), scale(frame_vec(t, 2), tan_quarter(sb))));
    return unit(p);
  }

  void connect() {
    for (int t = 0; t < 6; ++t)
      for (int s = 0; s < 4; ++s) {
        const Side& S = kSide[s];
        V3 a = point(t, n * S.ox, n * S.oy), b = point(t, n * S.ox + n * S.tx, n * S.oy + n * S.ty);
        nbr_tile[t][s] = -1;
        for (int t2 = 0; t2 < 6; ++t2) {
          if (t2 == t) continue;
          for (int s2 = 0; s2 < 4; ++s2) {
            const Side& Q = kSide[s2];
            V3 a2 = point(t2, n * Q.ox, n * Q.oy), b2 = point(t2, n * Q.ox + n * Q.tx, n * Q.oy + n * Q.ty);
            if (len(sub(a, a2)) < 1e-11 && len(sub(b, b2)) < 1e-11) {
              nbr_tile[t][s] = t2; nbr_side[t][s] = s2; nbr_flip[t][s] = false;
            } else if (len(sub(a, b2)) < 1e-11 && len(sub(b, a2)) < 1e-11) {
              nbr_tile[t][s] = t2; nbr_side[t][s] = s2; nbr_flip[t][s] = true;
            }
          }
        }
      }
  }

  // carry (X, Y) of tile t across side s (cube) or wrap it (periodic)
  void cross_side(int& t, double& X, double& Y, int s, Rot& R) const {
    if (!cubed) {
      const Side& S = kSide[s];
      X -= n * S.nx;  // periodic: shift by one period against the outward normal
      Y -= n * S.ny;
      return;
    }
    const Side& S = kSide[s];
    double rx = X - n * S.ox, ry = Y - n * S.oy;
    double along = rx * S.tx + ry * S.ty, depth = rx * S.nx + ry * S.ny;
    int t2 = nbr_tile[t][s], s2 = nbr_side[t][s];
    bool flip = nbr_flip[t][s];
    const Side& Q = kSide[s2];
    double along2 = flip ? n - along : along;
    X = n * Q.ox + along2 * Q.tx - depth * Q.nx;
    Y = n * Q.oy + along2 * Q.ty - depth * Q.ny;
    int sg = flip ? -1 : 1;
    Rot step;
    // e_x = tx*along_dir + nx*out_dir (orthonormal); along -> sg*along2, out -> -out2
    int ex = S.tx, eox = S.nx, ey = S.ty, eoy = S.ny;
    step.m[0][0] = ex * sg * Q.tx - eox * Q.nx;
    step.m[1][0] = ex * sg * Q.ty - eox * Q.ny;
    step.m[0][1] = ey * sg * Q.tx - eoy * Q.nx;
    step.m[1][1] = ey * sg * Q.ty - eoy * Q.ny;
    R = compose(step, R);
    t = t2;
  }
};

// role of the corner rotation: 0 along x (from the W/E strip), 1 along y
static void corner_turn(int n, int role, double& X, double& Y, Rot& R) {
  int ox = X < 0 ? -1 : 1, oy = Y < 0 ? -1 : 1;
  double cx = X < 0 ? 0.0 : n, cy = Y < 0 ? 0.0 : n;
  double da = ox * (X - cx), db = oy * (Y - cy);  // outward depths in x and y
  int s = ox * oy;
  Rot step;
  if (role == 0) {
    X = cx + ox * db;
    Y = cy - oy * da;
    step.m[0][0] = 0; step.m[1][0] = -s; step.m[0][1] = s; step.m[1][1] = 0;
  } else {
    X = cx - ox * db;
    Y = cy + oy * da;
    step.m[0][0] = 0; step.m[1][0] = s; step.m[0][1] = -s; step.m[1][1] = 0;
  }
  R = compose(step, R);
}

// Resolve the value-holding location of point (X, Y) of tile t.  role: corner
// role to use if the point is in a missing cube corner (-1: none -> NaN).
// Returns false for NaN.
static bool resolve(const Topology& T, int& t, double& X, double& Y, int role, Rot& R) {
  const int n = T.n;
  for (int it = 0; it < 8; ++it) {
    bool inx = X >= 0 && X <= n, iny = Y >= 0 && Y <= n;
    if (!inx && !iny) {
      if (!T.cubed) {  // periodic: both coordinates wrap
        X = X < 0 ? X + n : X - n;
        Y = Y < 0 ? Y + n : Y - n;
        continue;
      }
      if (role < 0) return false;
      corner_turn(n, role, X, Y, R);
      role = -1;
      continue;
    }
    if (!inx || !iny) {
      int s = X < 0 ? 0 : X > n ? 1 : Y < 0 ? 2 : 3;
      T.cross_side(t, X, Y, s, R);
      continue;
    }
    // inside or on a side line: a face on a side is owned by the lower tile
    // index (periodic: by the W / S side)
    int s = -1;
    if ((X == 0 || X == n) && Y > 0 && Y < n) s = X == 0 ? 0 : 1;
    if ((Y == 0 || Y == n) && X > 0 && X < n) s = Y == 0 ? 2 : 3;
    if (s < 0) return true;
    bool other_owns = T.cubed ? (T.nbr_tile[t][s] < t) : (s == 1 || s == 3);
    if (!other_owns) return true;
    T.cross_side(t, X, Y, s, R);
    return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// halo plans
// ---------------------------------------------------------------------------
// field kinds of a plan
//   CELL3 : cell scalar, strips of depth 3, cube-corner cells NaN
//   CELL1 : cell scalar, strips of depth 1 only
//   DGRID : vector pair, x-comp on y-faces (u), y-comp on x-faces (v); cube
//           corner x-faces from the y-turn, y-faces from the x-turn
//   CGRID : vector pair, x-comp on x-faces, y-comp on y-faces; corners NaN
//   LENGTH: unsigned face pair (lengths, sines); corners NaN
//   COSINE: face pair that takes the product of both basis signs
static void add_slot(const Topology& T, const Geo& g, int m, int t, int arr, int i, int j, int kind,
                     std::vector<HaloEntry>& out) {
  // arr: 0 cell, 1 x-face, 2 y-face
  double X = arr == 1 ? i : i + 0.5;
  double Y = arr == 2 ? j : j + 0.5;
  int role = -1;
  if (kind == K_DGRID) role = (arr == 1) ? 1 : 0;
  int ts = t;
  double Xs = X, Ys = Y;
  Rot R;
  HaloEntry e{};
  e.m = (short)m;
  e.dt = (unsigned char)t;
  e.dst = (int)pidx(g, j, i);
  e.flags = (unsigned char)(arr == 2 ? 1 : 0);
  bool ok = resolve(T, ts, Xs, Ys, role, R);
  if (ok && ts == t && Xs == X && Ys == Y) return;  // owns its value
  if (!ok) {
    e.sign = 0;
    e.src = 0;
    e.st = 0;
    out.push_back(e);
    return;
  }
  bool src_x = (Xs == std::floor(Xs)) && arr != 0;  // integer X: an x-face
  int si = (int)std::floor(Xs), sj = (int)std::floor(Ys);
  e.st = (unsigned char)ts;
  e.src = (int)pidx(g, sj, si);
  int sign = 1;
  if (arr != 0) {
    int comp;  // component stored in the destination slot
    if (kind == K_DGRID) comp = (arr == 1) ? 1 : 0;
    else comp = (arr == 1) ? 0 : 1;
    int ax, ay;
    R.image(comp, ax, ay);
    if (kind == K_DGRID || kind == K_CGRID) sign = ax + ay;
    if (kind == K_COSINE) {
      int bx, by, cx, cy;
      R.image(0, bx, by);
      R.image(1, cx, cy);
      sign = (bx + by) * (cx + cy);
    }
    if (!src_x) e.flags |= 2;
  }
  e.sign = (signed char)sign;
  out.push_back(e);
}

std::vector<HaloEntry> build_plan(const Topology& T, const Geo& g, int m, int kind) {
  std::vector<HaloEntry> out;
  const int n = g.n;
  const int d = (kind == K_CELL1) ? 1 : HALO;
  for (int t = 0; t < g.nt; ++t) {
    if (kind == K_CELL3 || kind == K_CELL1) {
      for (int j = -d; j < n + d; ++j)
        for (int i = -d; i < n + d; ++i) {
          bool inx = i >= 0 && i < n, iny = j >= 0 && j < n;
          if (inx && iny) continue;
          if (kind == K_CELL1 && !inx && !iny) continue;
          add_slot(T, g, m, t, 0, i, j, kind, out);
        }
      continue;
    }
    for (int j = -d; j < n + d; ++j)  // x-faces
      for (int i = -d; i <= n + d; ++i) {
        bool inside = i > 0 && i < n && j >= 0 && j < n;
        if (inside) continue;
        add_slot(T, g, m, t, 1, i, j, kind, out);
      }
    for (int j = -d; j <= n + d; ++j)  // y-faces
      for (int i = -d; i < n + d; ++i) {
        bool inside = i >= 0 && i < n && j > 0 && j < n;
        if (inside) continue;
        add_slot(T, g, m, t, 2, i, j, kind, out);
      }
  }
  return out;
}

// apply a plan to host planes of one member ([tile][plane], one level)
static void apply_plan_host(const std::vector<HaloEntry>& P, const Geo& g, double* xa, double* ya) {
  for (const HaloEntry& e : P) {
    double* dst = (e.flags & 1) ? ya : xa;
    const double* src = (e.flags & 2) ? ya : xa;
    double v = e.sign == 0 ? NAN : e.sign * src[(long long)e.st * g.plane + e.src];
    dst[(long long)e.dt * g.plane + e.dst] = v;
  }
}

// ---------------------------------------------------------------------------
// metric construction for one member
// ---------------------------------------------------------------------------
static double arc(V3 a, V3 b) { return std::atan2(len(cross(a, b)), dot(a, b)); }

static double excess(V3 a, V3 b, V3 c) {
  double num = std::fabs(dot(a, cross(b, c)));
  double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
  return 2.0 * std::atan2(num, den);
}

// unit tangent of the alpha (role 1) or beta (role 2) coordinate line at p
static V3 line_tangent(int t, V3 p, int r) {
  V3 a = frame_vec(t, r);
  return unit(sub(a, scale(p, dot(a, p))));
}

void build_metric(const GridSpec& spec, int m, const Geo& g, HostMetric& M, Plans& plans) {
  const int n = g.n, nt = g.nt;
  const long long P = g.plane;
  auto alloc = [&](std::vector<double>& v) { v.assign((size_t)(nt * P), NAN); };
  std::vector<double>* all[] = {&M.area, &M.rarea, &M.fA, &M.dx, &M.rdx, &M.dyc, &M.rdyc, &M.cosy, &M.siny,
                                &M.dy, &M.rdy, &M.dxc, &M.rdxc, &M.cosx, &M.sinx, &M.fC, &M.rareac};
  for (auto* v : all) alloc(*v);
  Topology T;
  T.n = n;
  T.cubed = spec.cubed;
  if (spec.cubed) T.connect();

  for (int kind = 0; kind < K_NUM; ++kind) plans.p[kind] = build_plan(T, g, m, kind);

  if (!spec.cubed) {
    const double h = spec.dx, a = h * h;
    for (int t = 0; t < nt; ++t)
      for (long long o = 0; o < P; ++o) {
        long long q = t * P + o;
        M.area[q] = a; M.rarea[q] = 1.0 / a; M.fA[q] = 0.0;
        M.dx[q] = h; M.rdx[q] = 1.0 / h; M.dyc[q] = h; M.rdyc[q] = 1.0 / h; M.cosy[q] = 0.0; M.siny[q] = 1.0;
        M.dy[q] = h; M.rdy[q] = 1.0 / h; M.dxc[q] = h; M.rdxc[q] = 1.0 / h; M.cosx[q] = 0.0; M.sinx[q] = 1.0;
        M.fC[q] = 0.0; M.rareac[q] = 1.0 / a;
      }
    M.da_min = a;
    return;
  }

  const double Rad = spec.radius, Om = spec.omega;
  // centre of cell (i, j) of tile t, the neighbour's for strip cells
  auto centre = [&](int t, int i, int j) {
    int ts = t;
    double X = i + 0.5, Y = j + 0.5;
    Rot R;
    resolve(T, ts, X, Y, -1, R);
    return T.point(ts, X, Y);
  };
  for (int t = 0; t < nt; ++t) {
    double* base;
    (void)base;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        V3 p0 = T.point(t, i, j), p1 = T.point(t, i + 1, j), p2 = T.point(t, i + 1, j + 1), p3 = T.point(t, i, j + 1);
        double A = (excess(p0, p1, p2) + excess(p0, p2, p3)) * Rad * Rad;
        long long q = t * P + pidx(g, j, i);
        M.area[q] = A;
        M.rarea[q] = 1.0 / A;
        M.fA[q] = 2.0 * Om * T.point(t, i + 0.5, j + 0.5).z;
      }
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i < n; ++i) {  // y-faces
        long long q = t * P + pidx(g, j, i);
        V3 a = T.point(t, i, j), b = T.point(t, i + 1, j);
        M.dx[q] = arc(a, b) * Rad;
        M.rdx[q] = 1.0 / M.dx[q];
        M.dyc[q] = arc(centre(t, i, j - 1), centre(t, i, j)) * Rad;
        M.rdyc[q] = 1.0 / M.dyc[q];
        V3 pm = T.point(t, i + 0.5, j);
        double c = dot(line_tangent(t, pm, 1), line_tangent(t, pm, 2));
        M.cosy[q] = c;
        M.siny[q] = std::sqrt(1.0 - c * c);
      }
    for (int j = 0; j < n; ++j)
      for (int i = 0; i <= n; ++i) {  // x-faces
        long long q = t * P + pidx(g, j, i);
        V3 a = T.point(t, i, j), b = T.point(t, i, j + 1);
        M.dy[q] = arc(a, b) * Rad;
        M.rdy[q] = 1.0 / M.dy[q];
        M.dxc[q] = arc(centre(t, i - 1, j), centre(t, i, j)) * Rad;
        M.rdxc[q] = 1.0 / M.dxc[q];
        V3 pm = T.point(t, i, j + 0.5);
        double c = dot(line_tangent(t, pm, 1), line_tangent(t, pm, 2));
        M.cosx[q] = c;
        M.sinx[q] = std::sqrt(1.0 - c * c);
      }
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {  // corners
        long long q = t * P + pidx(g, j, i);
        M.fC[q] = 2.0 * Om * T.point(t, i, j).z;
        bool corner = (i == 0 || i == n) && (j == 0 || j == n);
        double A;
        if (corner) {
          int ic = i == 0 ? 0 : n - 1, jc = j == 0 ? 0 : n - 1;
          int ix = i == 0 ? -1 : n, jy = j == 0 ? -1 : n;
          A = excess(centre(t, ic, jc), centre(t, ix, jc), centre(t, ic, jy)) * Rad * Rad;
        } else {
          V3 c00 = centre(t, i - 1, j - 1), c10 = centre(t, i, j - 1), c11 = centre(t, i, j), c01 = centre(t, i - 1, j);
          A = (excess(c00, c10, c11) + excess(c00, c11, c01)) * Rad * Rad;
        }
        M.rareac[q] = 1.0 / A;
      }
  }
  // halos of the metric by the same plans
  apply_plan_host(plans.p[K_CELL3], g, M.area.data(), M.area.data());
  apply_plan_host(plans.p[K_CELL3], g, M.rarea.data(), M.rarea.data());
  apply_plan_host(plans.p[K_CELL3], g, M.fA.data(), M.fA.data());
  apply_plan_host(plans.p[K_LENGTH], g, M.dy.data(), M.dx.data());
  apply_plan_host(plans.p[K_LENGTH], g, M.rdy.data(), M.rdx.data());
  apply_plan_host(plans.p[K_LENGTH], g, M.dxc.data(), M.dyc.data());
  apply_plan_host(plans.p[K_LENGTH], g, M.rdxc.data(), M.rdyc.data());
  apply_plan_host(plans.p[K_LENGTH], g, M.sinx.data(), M.siny.data());
  apply_plan_host(plans.p[K_COSINE], g, M.cosx.data(), M.cosy.data());
  double mn = INFINITY;
  for (int t = 0; t < nt; ++t)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) mn = std::min(mn, M.area[t * P + pidx(g, j, i)]);
  M.da_min = mn;
}

}  // namespace fv3
