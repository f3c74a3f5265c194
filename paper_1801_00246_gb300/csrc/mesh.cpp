// Host-side mesh setup: affine geometric factors (Section 5.2, Eq. operators2,
// elementOps), face connectivity, and the checks that guard every later launch.
#include <cstdlib>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "dg_internal.h"

namespace dgx {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(uint64_t(n), std::memory_order_relaxed); }

// Debug aid: with DG_POISON_SCRATCH=1 in the environment every scratch buffer
// the library allocates is filled with 0xFF bytes (NaN in FP32 and FP64), so a
// read of memory no kernel has written shows up as NaN instead of depending on
// what the allocator hands back; 2, 3 or 4 poison only the AMG, the solver
// workspace or the apply scratch.
cudaError_t poison(void* p, size_t bytes, int group) {
  static const int mode = [] {
    const char* v = std::getenv("DG_POISON_SCRATCH");
    return v ? std::atoi(v) : 0;
  }();
  if (mode == 0 || (mode != 1 && mode != group) || !p || bytes == 0) return cudaSuccess;
  return cudaMemset(p, 0xFF, bytes);
}
void set_error(const std::string& msg) { g_last_error = msg; }
std::mutex& table_mutex() {
  static std::mutex mu;
  return mu;
}
const char* last_error() { return g_last_error.c_str(); }

// Geometric factors per element: the affine map x = x0 + (x1-x0)(r+1)/2 +
// (x2-x0)(s+1)/2 has Jacobian [[x_r, x_s], [y_r, y_s]]; its inverse gives
// G^e = [[r_x, s_x], [r_y, s_y]] and J^e = x_r y_s - x_s y_r (must be > 0).
bool compute_geometry(dg_mesh* m, std::string& err) {
  const int64_t K = m->K;
  m->geo_h.resize(size_t(K) * 4);
  for (int64_t e = 0; e < K; ++e) {
    const int32_t* v = &m->EToV[3 * e];
    const double x0 = m->VX[v[0]], y0 = m->VY[v[0]];
    const double xr = 0.5 * (m->VX[v[1]] - x0), yr = 0.5 * (m->VY[v[1]] - y0);
    const double xs = 0.5 * (m->VX[v[2]] - x0), ys = 0.5 * (m->VY[v[2]] - y0);
    const double J = xr * ys - xs * yr;
    if (!(J > 0.0)) {
      err = "element " + std::to_string(e) + " has non-positive Jacobian (vertices not counter-clockwise?)";
      return false;
    }
    m->geo_h[4 * e + 0] = ys / J;   // r_x
    m->geo_h[4 * e + 1] = -yr / J;  // s_x
    m->geo_h[4 * e + 2] = -xs / J;  // r_y
    m->geo_h[4 * e + 3] = xr / J;   // s_y
  }
  return true;
}

// Face connectivity by sorting the (min, max) vertex pair of every face.
bool compute_connectivity(dg_mesh* m, const int8_t* bc, std::string& err) {
  const int64_t K = m->K;
  struct FaceKey {
    int32_t a, b;
    int64_t ef;
  };
  std::vector<FaceKey> keys(size_t(K) * 3);
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 3; ++f) {
      const int32_t va = m->EToV[3 * e + f], vb = m->EToV[3 * e + (f + 1) % 3];
      keys[3 * e + f] = {std::min(va, vb), std::max(va, vb), 3 * e + f};
    }
  std::sort(keys.begin(), keys.end(), [](const FaceKey& p, const FaceKey& q) {
    return p.a != q.a ? p.a < q.a : (p.b != q.b ? p.b < q.b : p.ef < q.ef);
  });
  m->conn_h.assign(size_t(K) * 3, 0);
  std::vector<char> matched(size_t(K) * 3, 0);
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].a == keys[i].a && keys[j].b == keys[i].b) ++j;
    if (j - i > 2) {
      err = "face shared by more than two elements";
      return false;
    }
    if (j - i == 2) {
      const int64_t p = keys[i].ef, q = keys[i + 1].ef;
      if ((p / 3) > (int64_t(1) << 29) || (q / 3) > (int64_t(1) << 29)) {
        err = "too many elements for the packed connectivity word";
        return false;
      }
      m->conn_h[p] = int32_t(((q / 3) << 2) | (q % 3));
      m->conn_h[q] = int32_t(((p / 3) << 2) | (p % 3));
      matched[p] = matched[q] = 1;
    }
    i = j;
  }
  for (int64_t ef = 0; ef < 3 * K; ++ef) {
    const int tag = bc ? bc[ef] : (matched[ef] ? 0 : 1);
    if (matched[ef]) {
      if (tag != 0) {
        err = "interior face " + std::to_string(ef) + " carries a boundary tag";
        return false;
      }
    } else {
      if (tag != 1 && tag != 2) {
        err = "boundary face " + std::to_string(ef) + " needs tag 1 (Dirichlet) or 2 (Neumann)";
        return false;
      }
      m->conn_h[ef] = -1 - tag;
    }
  }
  return true;
}

// Check that local face node j meets neighbour face node Nfp-1-j at the same
// physical point for every interior face (the orientation rule the kernels use).
bool check_face_matching(const dg_mesh* m, std::string& err) {
  const RefElem& R = m->ref[m->N];
  const int Nfp = R.Nfp;
  auto phys = [&](int64_t e, int node, double& x, double& y) {
    const int32_t* v = &m->EToV[3 * e];
    const double r = R.r[node], s = R.s[node];
    x = m->VX[v[0]] + 0.5 * (m->VX[v[1]] - m->VX[v[0]]) * (r + 1) + 0.5 * (m->VX[v[2]] - m->VX[v[0]]) * (s + 1);
    y = m->VY[v[0]] + 0.5 * (m->VY[v[1]] - m->VY[v[0]]) * (r + 1) + 0.5 * (m->VY[v[2]] - m->VY[v[0]]) * (s + 1);
  };
  for (int64_t e = 0; e < m->K; ++e)
    for (int f = 0; f < 3; ++f) {
      const int32_t c = m->conn_h[3 * e + f];
      if (c < 0) continue;
      const int64_t nb = c >> 2;
      const int fn = c & 3;
      const double h = std::sqrt(1.0 / std::fabs(m->geo_h[4 * e] * m->geo_h[4 * e + 3] -
                                                 m->geo_h[4 * e + 1] * m->geo_h[4 * e + 2]));
      for (int j = 0; j < Nfp; ++j) {
        double xa, ya, xb, yb;
        phys(e, R.fmask[f * Nfp + j], xa, ya);
        phys(nb, R.fmask[fn * Nfp + (Nfp - 1 - j)], xb, yb);
        if (std::hypot(xa - xb, ya - yb) > 1e-9 * h) {
          err = "face nodes of element " + std::to_string(e) + " face " + std::to_string(f) +
                " do not meet the neighbour's (non-conforming mesh?)";
          return false;
        }
      }
    }
  return true;
}

void node_coordinates(const dg_mesh* m, int degree, std::vector<double>& x, std::vector<double>& y) {
  const RefElem& R = m->ref[degree];
  x.resize(size_t(m->K) * R.Np);
  y.resize(size_t(m->K) * R.Np);
  for (int64_t e = 0; e < m->K; ++e) {
    const int32_t* v = &m->EToV[3 * e];
    for (int i = 0; i < R.Np; ++i) {
      const double r = R.r[i], s = R.s[i];
      x[size_t(e) * R.Np + i] = m->VX[v[0]] + 0.5 * (m->VX[v[1]] - m->VX[v[0]]) * (r + 1) +
                                0.5 * (m->VX[v[2]] - m->VX[v[0]]) * (s + 1);
      y[size_t(e) * R.Np + i] = m->VY[v[0]] + 0.5 * (m->VY[v[1]] - m->VY[v[0]]) * (r + 1) +
                                0.5 * (m->VY[v[2]] - m->VY[v[0]]) * (s + 1);
    }
  }
}

}  // namespace dgx
