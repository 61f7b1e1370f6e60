// Host-side plan construction in FP64: geometry, TDOA table, interpolation matrix rows,
// and the two offline fits of Sec. IV-A (low rank, Eq. min_Lambda_lr; sparse, Eq.
// min_Lambda_sp).  None of this runs per frame (Sec. IV-B: computed upfront).
#include "srp_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <thread>

namespace srp {

unsigned host_threads() {
  unsigned n = std::thread::hardware_concurrency();
  if (n == 0) n = 4;
  return std::min(n, 32u);
}

// Runs fn(begin, end) over [0, n) split into contiguous chunks, one per thread.
void parallel_for(long long n, const std::function<void(long long, long long)>& fn) {
  const unsigned T = host_threads();
  if (n <= 0) return;
  if (T <= 1 || n < 64) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> th;
  const long long chunk = (n + T - 1) / T;
  for (unsigned t = 0; t < T; ++t) {
    const long long b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back([&fn, b, e] { fn(b, e); });
  }
  for (auto& x : th) x.join();
}

// -----------------------------------------------------------------------------------
// Sec. II-A: pairs, distances, TDOAs; Eq. N_p: N_p = floor(d_p / c * fs) + N_aux.
// -----------------------------------------------------------------------------------
srp_status build_geometry(const srp_plan_desc& d, Geometry& g) {
  g.M = d.M;
  g.J = d.J;
  g.N = d.N;
  g.K = d.N / 2;
  g.fs = d.fs;
  g.c = d.c;
  g.pm.clear();
  g.pmp.clear();
  for (int mp = 0; mp < d.M - 1; ++mp)
    for (int m = mp + 1; m < d.M; ++m) {
      g.pm.push_back(m);
      g.pmp.push_back(mp);
    }
  g.P = static_cast<int>(g.pm.size());
  g.Np.assign(g.P, 0);
  g.off.assign(g.P, 0);
  int L = 0;
  for (int p = 0; p < g.P; ++p) {
    const double* a = d.mic_xyz + 3 * g.pm[p];
    const double* b = d.mic_xyz + 3 * g.pmp[p];
    const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
    g.Np[p] = static_cast<int>(std::floor(dist / d.c * d.fs)) + d.n_aux;
    if (g.Np[p] >= g.K) {
      set_error("N_p = " + std::to_string(g.Np[p]) + " >= K = " + std::to_string(g.K) +
                " for pair " + std::to_string(p) +
                ": the sample window is wider than the frame (increase N)");
      return SRP_EINVAL;
    }
    g.off[p] = L;
    L += 2 * g.Np[p] + 1;
  }
  g.L = L;
  // Eq. Deltat_i in samples: near field ((||r_m - q_i|| - ||r_m' - q_i||) / c) * fs;
  // far field ((r_m - r_m')^T q_i / c) * fs with q_i a unit incident direction.
  g.tau.assign(static_cast<size_t>(g.J) * g.P, 0.0);
  const int M = d.M;
  if (d.far_field) {
    parallel_for(g.J, [&](long long b, long long e) {
      for (long long i = b; i < e; ++i) {
        const double* q = d.grid_xyz + 3 * i;
        double* t = g.tau.data() + static_cast<size_t>(i) * g.P;
        for (int p = 0; p < g.P; ++p) {
          const double* a = d.mic_xyz + 3 * g.pm[p];
          const double* c = d.mic_xyz + 3 * g.pmp[p];
          t[p] = (((a[0] - c[0]) * q[0] + (a[1] - c[1]) * q[1] + (a[2] - c[2]) * q[2]) / d.c) * d.fs;
        }
      }
    });
    return SRP_OK;
  }
  parallel_for(g.J, [&](long long b, long long e) {
    std::vector<double> dist(M);
    for (long long i = b; i < e; ++i) {
      const double* q = d.grid_xyz + 3 * i;
      for (int m = 0; m < M; ++m) {
        const double* r = d.mic_xyz + 3 * m;
        const double dx = q[0] - r[0], dy = q[1] - r[1], dz = q[2] - r[2];
        dist[m] = std::sqrt(dx * dx + dy * dy + dz * dz);
      }
      double* t = g.tau.data() + static_cast<size_t>(i) * g.P;
      for (int p = 0; p < g.P; ++p) t[p] = ((dist[g.pm[p]] - dist[g.pmp[p]]) / d.c) * d.fs;
    }
  });
  return SRP_OK;
}

// Eq. Lambda_p: sinc(tau_p(i) - n), sinc(x) = sin(pi x)/(pi x), sinc(0) = 1.
static inline double sinc_pi(double x) {
  if (x == 0.0) return 1.0;
  const double y = M_PI * x;
  return std::sin(y) / y;
}

void lambda_row(const Geometry& g, int i, double* row) {
  const double* t = g.tau.data() + static_cast<size_t>(i) * g.P;
  for (int p = 0; p < g.P; ++p) {
    const int np = g.Np[p];
    double* r = row + g.off[p];
    for (int n = -np; n <= np; ++n) r[n + np] = sinc_pi(t[p] - static_cast<double>(n));
  }
}

// -----------------------------------------------------------------------------------
// Symmetric eigen-decomposition by the cyclic Jacobi method (rotations that annihilate
// one off-diagonal element at a time, Jacobi 1846 / Rutishauser's formulation).
// A: n x n row-major, destroyed.  V: eigenvectors as columns.  d: eigenvalues.
// -----------------------------------------------------------------------------------
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V,
                  std::vector<double>& d) {
  V.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[static_cast<size_t>(i) * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[static_cast<size_t>(p) * n + q] * A[static_cast<size_t>(p) * n + q];
    if (off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double& apq_ref = A[static_cast<size_t>(p) * n + q];
        const double apq = apq_ref;
        if (apq == 0.0) continue;
        const double app = A[static_cast<size_t>(p) * n + p];
        const double aqq = A[static_cast<size_t>(q) * n + q];
        const double gg = 100.0 * std::fabs(apq);
        if (sweep > 3 && std::fabs(app) + gg == std::fabs(app) &&
            std::fabs(aqq) + gg == std::fabs(aqq)) {
          apq_ref = 0.0;
          A[static_cast<size_t>(q) * n + p] = 0.0;
          continue;
        }
        const double theta = (aqq - app) / (2.0 * apq);
        double t = 1.0 / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        if (theta < 0) t = -t;
        const double c = 1.0 / std::sqrt(t * t + 1.0);
        const double s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double* rk = A.data() + static_cast<size_t>(k) * n;
          const double akp = rk[p], akq = rk[q];
          rk[p] = c * akp - s * akq;
          rk[q] = s * akp + c * akq;
        }
        double* rp = A.data() + static_cast<size_t>(p) * n;
        double* rq = A.data() + static_cast<size_t>(q) * n;
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = rp[k], aqk = rq[k];
          rp[k] = c * apk - s * aqk;
          rq[k] = s * apk + c * aqk;
        }
        rp[q] = 0.0;
        rq[p] = 0.0;
        for (int k = 0; k < n; ++k) {
          double* vk = V.data() + static_cast<size_t>(k) * n;
          const double vkp = vk[p], vkq = vk[q];
          vk[p] = c * vkp - s * vkq;
          vk[q] = s * vkp + c * vkq;
        }
      }
    }
  }
  d.resize(n);
  for (int i = 0; i < n; ++i) d[i] = A[static_cast<size_t>(i) * n + i];
}

// -----------------------------------------------------------------------------------
// Eq. min_Lambda_lr: Lambda_lr = Lambda V_R V_R^T with V_R the R leading eigenvectors
// of Lambda^T Lambda (its right singular vectors); tall = Lambda V_R, fat = V_R^T.
// -----------------------------------------------------------------------------------
srp_status fit_low_rank(const Geometry& g, int R, std::vector<float>& tall,
                        std::vector<float>& fat, std::vector<double>& sigma) {
  const int L = g.L, J = g.J;
  std::vector<double> G(static_cast<size_t>(L) * L, 0.0);
  // Gram matrix, parallel over its rows (each thread regenerates the Lambda rows it
  // needs in blocks of 64 and owns a strided set of Gram rows).
  const unsigned T = host_threads();
  {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < T; ++t) {
      th.emplace_back([&, t] {
        const int RB = 64;
        std::vector<double> blk(static_cast<size_t>(RB) * L);
        for (int i0 = 0; i0 < J; i0 += RB) {
          const int nb = std::min(RB, J - i0);
          for (int r = 0; r < nb; ++r) lambda_row(g, i0 + r, blk.data() + static_cast<size_t>(r) * L);
          for (int a = static_cast<int>(t); a < L; a += static_cast<int>(T)) {
            double* ga = G.data() + static_cast<size_t>(a) * L;
            for (int r = 0; r < nb; ++r) {
              const double* row = blk.data() + static_cast<size_t>(r) * L;
              const double va = row[a];
              if (va == 0.0) continue;
              for (int b = a; b < L; ++b) ga[b] += va * row[b];
            }
          }
        }
      });
    }
    for (auto& x : th) x.join();
  }
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < a; ++b) G[static_cast<size_t>(a) * L + b] = G[static_cast<size_t>(b) * L + a];
  std::vector<double> V, ev;
  jacobi_eigen(L, G, V, ev);
  std::vector<int> order(L);
  for (int i = 0; i < L; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
  sigma.resize(L);
  for (int i = 0; i < L; ++i) sigma[i] = std::sqrt(std::max(0.0, ev[order[i]]));
  const int Rp = (R + 7) / 8 * 8;  // padded rank (zero factors beyond R)
  std::vector<double> VR(static_cast<size_t>(L) * R);  // [L][R]
  for (int l = 0; l < L; ++l)
    for (int r = 0; r < R; ++r) VR[static_cast<size_t>(l) * R + r] = V[static_cast<size_t>(l) * L + order[r]];
  fat.assign(static_cast<size_t>(Rp) * L, 0.f);
  for (int r = 0; r < R; ++r)
    for (int l = 0; l < L; ++l) fat[static_cast<size_t>(r) * L + l] = static_cast<float>(VR[static_cast<size_t>(l) * R + r]);
  tall.assign(static_cast<size_t>(J) * Rp, 0.f);
  parallel_for(J, [&](long long b, long long e) {
    std::vector<double> row(L), acc(R);
    for (long long i = b; i < e; ++i) {
      lambda_row(g, static_cast<int>(i), row.data());
      std::fill(acc.begin(), acc.end(), 0.0);
      for (int l = 0; l < L; ++l) {
        const double v = row[l];
        const double* vr = VR.data() + static_cast<size_t>(l) * R;
        for (int r = 0; r < R; ++r) acc[r] += v * vr[r];
      }
      for (int r = 0; r < R; ++r) tall[static_cast<size_t>(i) * Rp + r] = static_cast<float>(acc[r]);
    }
  });
  return SRP_OK;
}

// -----------------------------------------------------------------------------------
// Eq. min_Lambda_sp: keep the nnz entries of largest magnitude.  Magnitudes are compared
// as integer keys round(|lambda| * 2^40); ties at the cut are taken in ascending
// (i, p, n) order, which is the row-major order of Lambda here.  Lambda is never stored.
//
// Window: |sinc(x)| <= 1 / (pi |x|), so every entry with |tau_p(i) - n| > W has a key of
// at most k_out(W) = key(1 / (pi W)).  Selecting among the entries inside the window
// (a subset) gives a cut key k_W <= the true cut; when k_out(W) + 2 < k_W no entry outside
// the window can reach the cut and the selection inside the window is exact (ties
// included: they all carry the key k_W and lie inside).  Otherwise W doubles, up to the
// whole of Lambda.  The window makes the cost O(J P W) instead of O(J L).
// Selection inside the window: histogram of key >> 24, exact cut inside the bucket,
// per-row counts, fill -- all in parallel over rows.
// -----------------------------------------------------------------------------------
static inline uint64_t sparse_key(double v) {
  return static_cast<uint64_t>(std::floor(std::fabs(v) * 1099511627776.0 + 0.5));  // 2^40
}

// Calls fn(l, value) for the entries of row i with |tau_p(i) - n| <= W (all when W < 0),
// in ascending column order.
template <typename Fn>
static inline void window_row(const Geometry& g, int i, double W, Fn&& fn) {
  const double* t = g.tau.data() + static_cast<size_t>(i) * g.P;
  for (int p = 0; p < g.P; ++p) {
    const int np = g.Np[p];
    int n0 = -np, n1 = np;
    if (W >= 0) {
      n0 = std::max(n0, static_cast<int>(std::ceil(t[p] - W)));
      n1 = std::min(n1, static_cast<int>(std::floor(t[p] + W)));
    }
    for (int n = n0; n <= n1; ++n) {
      const double x = t[p] - static_cast<double>(n);
      fn(g.off[p] + n + np, sinc_pi(x));
    }
  }
}

srp_status fit_sparse(const Geometry& g, long long nnz, std::vector<long long>& row_ptr,
                      std::vector<int>& col, std::vector<float>& val, long long& tied) {
  const int J = g.J;
  const int SHIFT = 24;
  const size_t NB = (size_t(1) << 16) + 2;
  const unsigned T = host_threads();
  int maxNp = 0;
  for (int p = 0; p < g.P; ++p) maxNp = std::max(maxNp, g.Np[p]);
  for (double W = 8.0;; W *= 2.0) {
    const bool full = W > 2.0 * maxNp + 2.0;  // the window covers every lag
    const double Wuse = full ? -1.0 : W;
    // pass 1: histogram of the top key bits (and the candidate count)
    std::vector<std::vector<long long>> hist(T, std::vector<long long>(NB, 0));
    {
      std::vector<std::thread> th;
      const long long chunk = (J + T - 1) / T;
      for (unsigned t = 0; t < T; ++t)
        th.emplace_back([&, t] {
          const long long b = t * chunk, e = std::min<long long>(J, b + chunk);
          for (long long i = b; i < e; ++i)
            window_row(g, static_cast<int>(i), Wuse,
                       [&](int, double v) { hist[t][sparse_key(v) >> SHIFT]++; });
        });
      for (auto& x : th) x.join();
    }
    std::vector<long long> H(NB, 0);
    long long cand = 0;
    for (unsigned t = 0; t < T; ++t)
      for (size_t b = 0; b < NB; ++b) H[b] += hist[t][b];
    hist.clear();
    for (size_t b = 0; b < NB; ++b) cand += H[b];
    if (cand < nnz) {
      if (full) {
        set_error("internal: fewer entries than Q_Lambda");
        return SRP_EINVAL;
      }
      continue;
    }
    long long above = 0;
    size_t bstar = NB - 1;
    for (size_t b = NB; b-- > 0;) {
      if (above + H[b] >= nnz) {
        bstar = b;
        break;
      }
      above += H[b];
    }
    // pass 2: exact cut inside bucket bstar
    std::vector<std::vector<uint64_t>> inb_t(T);
    {
      std::vector<std::thread> th;
      const long long chunk = (J + T - 1) / T;
      for (unsigned t = 0; t < T; ++t)
        th.emplace_back([&, t] {
          const long long b = t * chunk, e = std::min<long long>(J, b + chunk);
          for (long long i = b; i < e; ++i)
            window_row(g, static_cast<int>(i), Wuse, [&](int, double v) {
              const uint64_t k = sparse_key(v);
              if ((k >> SHIFT) == bstar) inb_t[t].push_back(k);
            });
        });
      for (auto& x : th) x.join();
    }
    std::vector<uint64_t> inb;
    inb.reserve(static_cast<size_t>(H[bstar]));
    for (auto& v : inb_t) inb.insert(inb.end(), v.begin(), v.end());
    inb_t.clear();
    const long long need_in_bucket = nnz - above;  // >= 1
    std::nth_element(inb.begin(), inb.begin() + (inb.size() - need_in_bucket), inb.end());
    const uint64_t kth = inb[inb.size() - need_in_bucket];
    if (!full) {
      const uint64_t k_out = sparse_key(1.0 / (M_PI * W));
      if (k_out + 2 >= kth) continue;  // an entry outside the window could reach the cut
    }
    long long gt_in_bucket = 0, eq = 0;
    for (uint64_t k : inb) {
      gt_in_bucket += (k > kth);
      eq += (k == kth);
    }
    inb.clear();
    inb.shrink_to_fit();
    const long long take_ties = need_in_bucket - gt_in_bucket;
    tied = eq;
    // pass 3: per-row counts, then fill in row order with the tie budget
    std::vector<int> cnt_gt(J, 0), cnt_eq(J, 0);
    parallel_for(J, [&](long long b, long long e) {
      for (long long i = b; i < e; ++i) {
        int a = 0, q = 0;
        window_row(g, static_cast<int>(i), Wuse, [&](int, double v) {
          const uint64_t k = sparse_key(v);
          a += (k > kth);
          q += (k == kth);
        });
        cnt_gt[i] = a;
        cnt_eq[i] = q;
      }
    });
    std::vector<int> ties_row(J, 0);
    long long budget = take_ties;
    row_ptr.assign(static_cast<size_t>(J) + 1, 0);
    for (int i = 0; i < J; ++i) {
      const int tk = static_cast<int>(std::min<long long>(budget, cnt_eq[i]));
      ties_row[i] = tk;
      budget -= tk;
      row_ptr[i + 1] = row_ptr[i] + cnt_gt[i] + tk;
    }
    if (row_ptr[J] != nnz) {
      set_error("internal: sparse selection count mismatch");
      return SRP_EINVAL;
    }
    col.assign(static_cast<size_t>(nnz), 0);
    val.assign(static_cast<size_t>(nnz), 0.f);
    parallel_for(J, [&](long long b, long long e) {
      for (long long i = b; i < e; ++i) {
        long long w = row_ptr[i];
        int ties = ties_row[i];
        window_row(g, static_cast<int>(i), Wuse, [&](int l, double v) {
          const uint64_t k = sparse_key(v);
          bool keep = k > kth;
          if (!keep && k == kth && ties > 0) {
            keep = true;
            --ties;
          }
          if (keep) {
            col[w] = l;
            val[w] = static_cast<float>(v);
            ++w;
          }
        });
      }
    });
    return SRP_OK;
  }
}

}  // namespace srp
