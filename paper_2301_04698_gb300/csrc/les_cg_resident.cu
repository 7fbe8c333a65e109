// les_cg_resident.cu -- the conjugate-gradient Poisson solve with its
// vectors resident in shared memory (Sec. 2.4: L_c psi = b, compact 7-point
// Laplacian, periodic in x, y, mirror or periodic in z; mean of b removed,
// psi returned with zero mean).
//
// When the whole grid fits in the GPU's shared memory (a 128 x 128 x 96 FP32
// grid needs about 27 MB of the 34 MB on 152 SMs), every iteration of the
// streaming solver is dominated by the latency of its passes through L2, not
// by their bytes.  Here each block of one persistent cooperative launch owns
// a brick of bx x by x bz nodes for the whole solve and keeps x, r, p and
// q = L_c p of its brick (p with a one-node ghost layer) in shared memory.  The only
// global traffic of an iteration is the exchange of brick faces:
//   phase A  p = r + beta p in place; the ghost layer is filled from the
//            neighbours' published faces of r (this iteration) and p (the
//            previous one, double-buffered by parity) as r + beta p_old, so
//            no barrier separates the p update from the matvec; p faces
//            published; q = L_c p; p.q
//   phase B  x += alpha p, r -= alpha q; r faces published; r.r
// each followed by a grid-wide sum (les_gridsync.cuh; FP32 dot products are
// accumulated as compensated FP32 pairs, FP64 ones in FP64).  The p_old
// faces are copied into the ghost layer asynchronously while the second grid
// sum is in flight, so that after it only the r faces are loaded, in one
// batch whose latency overlaps the end of the iteration in thread 0 (beta
// and the convergence test) and the owned update.
#include <algorithm>
#include <string>
#include <type_traits>

#include "les_gridsync.cuh"
#include "les_internal.h"

namespace les {
namespace {

constexpr int kResThreads = 512;

template <typename T>
struct ResArgs {
  int nx, ny, nz, walls;
  T cx, cy, cz;      // 1/dx^2, 1/dy^2, 1/dz^2
  int by, bz;        // brick extent in y and z (x extent: the template BX)
  int px, py;        // bricks along x and y
  long long n;
  const T* b;
  T* x;
  T* rg;             // published faces of r
  T* pg0;            // published faces of p, even iterations
  T* pg1;            // ... odd iterations
  double* partials;  // [4][gridDim.x]
  FusedBar* bar;
  SolverCtl* ctl;
  double tol;
  int maxit;
  long long spin_cycles;
  unsigned expected;
  int guard;
};

__device__ __forceinline__ int zghost(int k, int nz, int walls) {
  if (walls) return k < 0 ? -1 - k : (k >= nz ? 2 * nz - 1 - k : k);
  return k < 0 ? k + nz : (k >= nz ? k - nz : k);
}

template <typename T, int BX>
__global__ void __launch_bounds__(kResThreads, 1) k_cg_resident(ResArgs<T> f) {
  constexpr int L = BX / 32;  // nodes per lane along a brick row
  // ghost rows per warp (and x-face ghosts per thread) whose loads are in
  // flight together, within the registers
  constexpr int RB = sizeof(T) == 4 ? (L >= 4 ? 3 : 4) : (L >= 2 ? 1 : 2);
  constexpr int XB = sizeof(T) == 4 ? 4 : 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int by = f.by, bz = f.bz;
  const int SY = BX + 2, SZ = (BX + 2) * (by + 2);  // strides of the haloed p brick
  const int nrow = by * bz;
  const int bcells = BX * nrow;
  T* P = reinterpret_cast<T*>(smraw);  // (BX + 2)(by + 2)(bz + 2)
  T* R = P + SZ * (bz + 2);            // BX by bz
  T* X = R + bcells;                   // BX by bz
  T* Q = X + bcells;                   // BX by bz: L_c p of this iteration
  // per brick row: P offset | face bit, global offset (8-byte aligned: the
  // T arrays above hold an even number of elements)
  int2* ROWS = reinterpret_cast<int2*>(Q + bcells);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  const int bi = blockIdx.x % f.px, bj = (blockIdx.x / f.px) % f.py, bk = blockIdx.x / (f.px * f.py);
  const int i0 = bi * BX, j0 = bj * by, k0 = bk * bz;
  const T cx = f.cx, cy = f.cy, cz = f.cz;

  // global index of local node (lx, ly, lz), at most one node outside the brick
  auto gidx = [&](int lx, int ly, int lz) -> size_t {
    int i = i0 + lx, j = j0 + ly;
    i = i < 0 ? i + f.nx : (i >= f.nx ? i - f.nx : i);
    j = j < 0 ? j + f.ny : (j >= f.ny ? j - f.ny : j);
    const int k = zghost(k0 + lz, f.nz, f.walls);
    return ((size_t)k * f.ny + j) * f.nx + i;
  };
  // second differences formed before scaling: for smooth p they are small
  // differences of nearly equal values, exact in floating point
  auto Lc = [&](int pi) -> T {
    const T c2 = T(2) * P[pi];
    return (P[pi - 1] + P[pi + 1] - c2) * cx + (P[pi - SY] + P[pi + SY] - c2) * cy +
           (P[pi - SZ] + P[pi + SZ] - c2) * cz;
  };
  // A brick spanning the periodic x extent is its own x neighbour: its x
  // ghosts are copies of its own end nodes, written with them, and its x
  // faces are not published.
  const bool xself = f.px == 1;
  // body(c, pi, g, face) for every owned node: c its index in R / X, pi in P,
  // g in global memory; face: the node lies on a brick surface that a
  // neighbour reads
  // the row table: row index arithmetic once per launch, not once per pass
  const size_t gbase = ((size_t)k0 * f.ny + j0) * f.nx + i0;
  for (int row = tid; row < nrow; row += nthr) {
    const int ly = row % by, lz = row / by;
    const bool rface = ly == 0 || ly == by - 1 || lz == 0 || lz == bz - 1;
    const int prow = (lz + 1) * SZ + (ly + 1) * SY + 1;
    ROWS[row] = make_int2(prow | (rface ? (int)0x80000000u : 0), (lz * f.ny + ly) * f.nx);
  }
  __syncthreads();
  // store p at owned node (c, pi), and at its periodic x image in the ghost
  // layer for a brick that is its own x neighbour
  auto put_p = [&](int c, int pi, T v) {
    P[pi] = v;
    if (xself) {
      const int lx = c & (BX - 1);
      if (lx == 0) P[pi + BX] = v;
      else if (lx == BX - 1) P[pi - BX] = v;
    }
  };
  auto own = [&](auto&& body) {
    for (int row = warp; row < nrow; row += nwarp) {
      const int2 t = ROWS[row];
      const bool rface = t.x < 0;
      const int prow = t.x & 0x7fffffff;
      const size_t grow = gbase + (unsigned)t.y;
#pragma unroll
      for (int u = 0; u < L; ++u) {
        const int lx = lane + 32 * u;
        body(row * BX + lx, prow + lx, grow + lx, rface || (!xself && (lx == 0 || lx == BX - 1)));
      }
    }
  };
  // fill the ghost layer of P with a, or with a + coef P where the ghost
  // layer already holds a staged second operand (stage() below), for each
  // face-neighbour node outside the brick (edges and corners are not used by
  // the 7-point stencil).  Rows along x: the two z faces (2 by rows), then
  // the two y faces (2 bz rows); the two x faces are strided single nodes.
  // Every load of a batch is issued before any loaded value is used, so a
  // batch costs one round of memory latency; when one batch per thread covers
  // all ghosts, between() runs while the loads are in flight, and coef is
  // read after it (between() may set it and must make the staged operand
  // visible block-wide).
  const int nr = 2 * by + 2 * bz;
  const int nxg = xself ? 0 : 2 * nrow;  // x-face ghosts loaded from neighbours
  const bool one_round = nr <= RB * nwarp && nxg <= XB * nthr;
  auto ghost_row = [&](int row, int& ly, int& lz) {
    if (row < 2 * by) {
      ly = row >> 1;
      lz = (row & 1) ? bz : -1;
    } else {
      lz = (row - 2 * by) >> 1;
      ly = (row & 1) ? by : -1;
    }
  };
  auto ghosts = [&](auto two, const T* A, const T& coef, auto&& between) {
    constexpr bool TWO = decltype(two)::value;
    if (one_round) {
      T va[RB][L], xa[XB];
      int pr[RB], xpi[XB];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int row = warp + q * nwarp;
        pr[q] = -1;
        if (row < nr) {
          int ly, lz;
          ghost_row(row, ly, lz);
          pr[q] = (lz + 1) * SZ + (ly + 1) * SY + 1;
          const size_t g0 = gidx(0, ly, lz);
#pragma unroll
          for (int u = 0; u < L; ++u) {
            va[q][u] = __ldcg(A + g0 + lane + 32 * u);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < XB; ++q) {
        const int c = tid + q * nthr;
        xpi[q] = -1;
        if (c < nxg) {
          const int row = c >> 1, ly = row % by, lz = row / by, lx = (c & 1) ? BX : -1;
          xpi[q] = (lz + 1) * SZ + (ly + 1) * SY + 1 + lx;
          const size_t g = gidx(lx, ly, lz);
          xa[q] = __ldcg(A + g);
        }
      }
      between();
      const T cf = coef;
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (pr[q] >= 0)
#pragma unroll
          for (int u = 0; u < L; ++u) {
            T& d = P[pr[q] + lane + 32 * u];
            if constexpr (TWO) d = va[q][u] + cf * d;
            else d = va[q][u];
          }
#pragma unroll
      for (int q = 0; q < XB; ++q)
        if (xpi[q] >= 0) {
          if constexpr (TWO) P[xpi[q]] = xa[q] + cf * P[xpi[q]];
          else P[xpi[q]] = xa[q];
        }
      return;
    }
    between();
    const T cf = coef;
    for (int r0 = warp; r0 < nr; r0 += RB * nwarp) {
      T va[RB][L];
      int pr[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int row = r0 + q * nwarp;
        pr[q] = -1;
        if (row < nr) {
          int ly, lz;
          ghost_row(row, ly, lz);
          pr[q] = (lz + 1) * SZ + (ly + 1) * SY + 1;
          const size_t g0 = gidx(0, ly, lz);
#pragma unroll
          for (int u = 0; u < L; ++u) {
            va[q][u] = __ldcg(A + g0 + lane + 32 * u);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (pr[q] >= 0)
#pragma unroll
          for (int u = 0; u < L; ++u) {
            T& d = P[pr[q] + lane + 32 * u];
            if constexpr (TWO) d = va[q][u] + cf * d;
            else d = va[q][u];
          }
    }
    for (int c0 = tid; c0 < nxg; c0 += XB * nthr) {
      T xa[XB];
      int pi[XB];
#pragma unroll
      for (int q = 0; q < XB; ++q) {
        const int c = c0 + q * nthr;
        pi[q] = -1;
        if (c < nxg) {
          const int row = c >> 1, ly = row % by, lz = row / by, lx = (c & 1) ? BX : -1;
          pi[q] = (lz + 1) * SZ + (ly + 1) * SY + 1 + lx;
          const size_t g = gidx(lx, ly, lz);
          xa[q] = __ldcg(A + g);
        }
      }
#pragma unroll
      for (int q = 0; q < XB; ++q)
        if (pi[q] >= 0) {
          if constexpr (TWO) P[pi[q]] = xa[q] + cf * P[pi[q]];
          else P[pi[q]] = xa[q];
        }
    }
  };
  auto nothing = [] {};
  // stage B at every ghost node into P's ghost layer with asynchronous copies
  // (one commit group), spread over warps w = 0 .. nw-1 of the caller's
  // choosing; the caller waits for the group and synchronises the block
  // before the ghosts are read
  auto stage = [&](const T* B, int w, int nw) {
    for (int row = w; row < nr; row += nw) {
      int ly, lz;
      ghost_row(row, ly, lz);
      const int pr = (lz + 1) * SZ + (ly + 1) * SY + 1;
      const size_t g0 = gidx(0, ly, lz);
#pragma unroll
      for (int u = 0; u < L; ++u) cp_async(P + pr + lane + 32 * u, B + g0 + lane + 32 * u);
    }
    for (int c = 32 * w + lane; c < nxg; c += 32 * nw) {
      const int row = c >> 1, ly = row % by, lz = row / by, lx = (c & 1) ? BX : -1;
      cp_async(P + (lz + 1) * SZ + (ly + 1) * SY + 1 + lx, B + gidx(lx, ly, lz));
    }
    cp_commit();
  };

  GridSync gs{f.bar, f.partials, f.spin_cycles, f.expected, 0u};
  // The scalar recurrences of CG run in thread 0 (FP64 division and square
  // root are long instruction sequences on this GPU); thread 0 broadcasts
  // the status and the FP32/FP64 coefficients through shared memory.
  __shared__ struct {
    T ta, tb, mean;
    int status, restart;
  } sc;
  double rr = 0.0, bb = 0.0, rel = 0.0, beta = 0.0;  // meaningful in thread 0
  int status = 0;  // 0 running, 1 converged, 2 maxit, 3 breakdown, 4 zero rhs, 5 timeout
  // mean of b; b staged in R
  {
    Dot<T> a1[1];
    own([&](int c, int, size_t g, bool) {
      const T v = __ldcg(f.b + g);
      R[c] = v;
      a1[0].add(v);
    });
    double t[1];
    const bool ok = grid_dot_t0<1>(a1, gs, t);
    if (tid == 0) {
      sc.status = ok ? 0 : 5;
      sc.mean = (T)(t[0] / (double)f.n);
    }
    __syncthreads();
    status = sc.status;
  }
  const T mean = sc.mean;

  // x0 with its ghosts; r = (b - mean) - L_c x0, published; r.r and |b - mean|^2
  if (!status) {
    own([&](int c, int pi, size_t g, bool) {
      const T v = __ldcg(f.x + g);
      X[c] = v;
      put_p(c, pi, v);
    });
    const T one = T(1);
    ghosts(std::false_type{}, f.x, one, nothing);
    __syncthreads();
    Dot<T> a2[2];
    own([&](int c, int pi, size_t g, bool face) {
      const T bm = R[c] - mean;
      const T rv = bm - Lc(pi);
      R[c] = rv;
      if (face) __stcg(f.rg + g, rv);
      a2[0].add(rv * rv);
      a2[1].add(bm * bm);
    });
    double s2[2];
    const bool ok = grid_dot_t0<2>(a2, gs, s2);
    if (tid == 0) {
      // the plain solver judges a learned first guess: if it leaves a larger
      // residual than x0 = 0, restart from zero (r = b - mean b, r.r = |b|^2)
      sc.status = ok ? 0 : 5;
      sc.restart = ok && f.guard && s2[0] > s2[1];
      rr = sc.restart ? s2[1] : s2[0];
      bb = s2[1];
    }
    __syncthreads();
    status = sc.status;
    if (!status && sc.restart) {
      own([&](int c, int, size_t g, bool face) {
        const T rv = __ldcg(f.b + g) - mean;
        X[c] = T(0);
        R[c] = rv;
        if (face) __stcg(f.rg + g, rv);
      });
      Dot<T> none[1];
      double t[1];
      const bool ok2 = grid_dot_t0<1>(none, gs, t);  // a grid barrier: the new faces are visible
      if (tid == 0) sc.status = ok2 ? 0 : 5;
      __syncthreads();
      status = sc.status;
    }
  }
  if (tid == 0) {
    if (!status) {
      if (bb == 0.0) status = 4;
      else {
        rel = sqrt(rr / bb);
        if (rel <= f.tol) status = 1;
        else if (f.maxit <= 0) status = 2;
      }
    }
    sc.status = status;
  }
  __syncthreads();
  status = sc.status;

  // convergence: |r| <= tol |b - mean| tested as r.r <= tol^2 |b - mean|^2,
  // so that no square root sits between two iterations
  const double rr_stop = f.tol * f.tol * bb;  // meaningful in thread 0
  int iter = 0;
  T tb = T(0);
  double rr_new = 0.0;  // thread 0: r.r of the grid sum that closed the last iteration
  bool sum_ok = true;   // thread 0: that grid sum completed
  // the end of an iteration in thread 0 (beta, convergence, status),
  // broadcast to the block
  auto close_iter = [&] {
    if (tid == 0) {
      if (!sum_ok) {
        status = 5;
      } else {
        beta = rr_new / rr;
        rr = rr_new;
        if (rr_new <= rr_stop) status = 1;
        else if (iter >= f.maxit) status = 2;
        else if (!isfinite(rr_new)) status = 3;
        sc.tb = (T)beta;
      }
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
    tb = sc.tb;
  };
  if (!status) {
    for (;;) {
      const bool first = iter == 0;
      // this iteration's p faces; the previous iteration's (the other parity)
      // may still be in flight to a neighbour's ghost layer until the next
      // grid sum
      T* pw = (iter & 1) ? f.pg1 : f.pg0;
      // phase A: p = r + beta p (owned in place, ghosts from published faces
      // as r + beta p_old, p_old staged in the ghost layer while the previous
      // grid sum was in flight).  The loads of r are issued first; while they
      // are in flight thread 0 closes the previous iteration (beta, status)
      // and the block updates its owned nodes.
      auto update = [&] {
        if (!first) {
          cp_wait<0>();  // the staged p_old; close_iter's barrier shares it
          close_iter();
        }
        if (status) return;
        own([&](int c, int pi, size_t g, bool face) {
          const T pv = first ? R[c] : R[c] + tb * P[pi];
          put_p(c, pi, pv);
          if (face) __stcg(pw + g, pv);
        });
      };
      if (first) ghosts(std::false_type{}, f.rg, tb, update);
      else ghosts(std::true_type{}, f.rg, tb, update);
      if (status) break;  // the ghosts just written are not used
      __syncthreads();
      Dot<T> apq[1];
      own([&](int c, int pi, size_t, bool) {
        const T qv = Lc(pi);
        Q[c] = qv;
        apq[0].add(P[pi] * qv);
      });
      {
        double t[1];
        const bool ok = grid_dot_t0<1>(apq, gs, t);
        if (tid == 0) {
          const double pq = t[0];
          if (!ok) status = 5;
          else if (pq == 0.0 || !isfinite(pq)) status = 3;
          else sc.ta = (T)(rr / pq);
          sc.status = status;
        }
        __syncthreads();
        status = sc.status;
        if (status) break;
      }
      const T ta = sc.ta;
      // phase B: x += alpha p, r -= alpha q, r faces published, r.r
      Dot<T> ar[1];
      own([&](int c, int pi, size_t g, bool face) {
        const T pv = P[pi];
        X[c] += ta * pv;
        const T rv = R[c] - ta * Q[c];
        R[c] = rv;
        if (face) __stcg(f.rg + g, rv);
        ar[0].add(rv * rv);
      });
      // while the grid sum is in flight (after this block's release), warps
      // 1.. stage this iteration's p faces -- complete everywhere since the
      // previous grid sum -- into the ghost layer for the next phase A
      double t[1];
      const bool ok = grid_dot_t0<1>(ar, gs, t, [&](int w, int nw) { stage(pw, w, nw); });
      iter += 1;
      if (tid == 0) {
        sum_ok = ok;
        rr_new = t[0];
      }
      // the grid sum has completed (or timed out, which close_iter reports):
      // from here every thread may read the faces the other blocks published
      __syncthreads();
    }
  }
  cp_wait<0>();  // no staging copy outlives the loop
  if (tid == 0 && iter > 0 && bb > 0.0) rel = sqrt(rr / bb);

  // zero-mean gauge (or zero for a zero right side), written back to x
  if (status != 5) {
    Dot<T> ax[1];
    own([&](int c, int, size_t, bool) { ax[0].add(X[c]); });
    double t[1];
    const bool ok = grid_dot_t0<1>(ax, gs, t);
    if (tid == 0) {
      if (!ok) status = 5;
      sc.mean = (T)(t[0] / (double)f.n);
      sc.status = status;
    }
    __syncthreads();
    status = sc.status;
    if (status != 5) {
      const T mx = sc.mean;
      own([&](int c, int, size_t g, bool) { __stcg(f.x + g, status == 4 ? T(0) : X[c] - mx); });
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    f.ctl->iter = iter;
    f.ctl->rel = rel;
    f.ctl->done = status;
  }
}

struct Plan {
  int bx = 0, by = 0, bz = 0, px = 0, py = 0, pz = 0;
  size_t smem = 0;
};

template <typename T>
size_t resident_smem(int bx, int by, int bz) {
  return ((size_t)(bx + 2) * (by + 2) * (bz + 2) + 3 * (size_t)bx * by * bz) * sizeof(T) +
         (size_t)by * bz * sizeof(int2);
}

// Brick decomposition: bx in {128, 64, 32} dividing nx, by | ny, bz | nz,
// at most one brick per SM and within the per-block shared memory; among
// those the one with the least work per block (owned nodes + ghost nodes +
// a per-block barrier cost).
template <typename T>
bool make_plan(const Grid<T>& g, int nsm, size_t smem_max, int max_blocks, Plan& best) {
  long long best_score = -1;
  const int gmax = std::min(nsm, max_blocks);
  for (int bx : {128, 64, 32}) {
    if (g.nx % bx) continue;
    for (int by = 1; by <= g.ny; ++by) {
      if (g.ny % by) continue;
      for (int bz = 1; bz <= g.nz; ++bz) {
        if (g.nz % bz) continue;
        const long long G = (long long)(g.nx / bx) * (g.ny / by) * (g.nz / bz);
        if (G > gmax) continue;
        const size_t smem = resident_smem<T>(bx, by, bz);
        if (smem > smem_max) continue;
        const long long cells = (long long)bx * by * bz;
        // x-face ghosts are strided single nodes, one 32-byte sector each:
        // weighted as eight; a brick as wide as the grid loads none
        const long long ghosts = 2LL * bx * by + 2LL * bx * bz + (bx == g.nx ? 0LL : 16LL * by * bz);
        const long long score = cells + ghosts + 4 * G;
        if (best_score < 0 || score < best_score) {
          best_score = score;
          best.bx = bx;
          best.by = by;
          best.bz = bz;
          best.px = g.nx / bx;
          best.py = g.ny / by;
          best.pz = g.nz / bz;
          best.smem = smem;
        }
      }
    }
  }
  return best_score >= 0;
}

template <typename T>
const void* resident_kernel(int bx) {
  switch (bx) {
    case 128: return (const void*)k_cg_resident<T, 128>;
    case 64: return (const void*)k_cg_resident<T, 64>;
    case 32: return (const void*)k_cg_resident<T, 32>;
    default: return nullptr;
  }
}

}  // namespace

template <typename T>
int poisson_solve_resident(const SolverArgs<T>& a, const FusedCfg& fc, const T* b, T* x, double tol, int maxit,
                           int* iters, double* rel, std::string* err, bool* used) {
  *used = false;
  if (!(a.op == LES_OP_COMPACT && a.solver == LES_SOLVER_CG && a.g.nz >= 2 && a.bar && a.r && a.p0 && a.p1))
    return LES_OK;
  int dev = 0, nsm = 0, smem_optin = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) {
    if (err) *err = std::string("resident CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  Plan pl;
  // leave room for the reductions' static shared memory (about 1 KB)
  if (!make_plan(a.g, nsm, (size_t)std::max(0, smem_optin - 2048), fc.max_blocks, pl)) return LES_OK;
  const void* kern = resident_kernel<T>(pl.bx);
  int per_sm = 0;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kResThreads, pl.smem)) != cudaSuccess) {
    if (err) *err = std::string("resident CG occupancy: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const long long G = (long long)pl.px * pl.py * pl.pz;
  if (per_sm < 1 || G > (long long)per_sm * nsm) return LES_OK;  // not co-resident: stream instead
  ResArgs<T> f;
  f.nx = a.g.nx;
  f.ny = a.g.ny;
  f.nz = a.g.nz;
  f.walls = a.g.walls;
  f.cx = a.g.idx * a.g.idx;
  f.cy = a.g.idy * a.g.idy;
  f.cz = a.g.idz * a.g.idz;
  f.by = pl.by;
  f.bz = pl.bz;
  f.px = pl.px;
  f.py = pl.py;
  f.n = (long long)f.nx * f.ny * f.nz;
  f.b = b;
  f.x = x;
  f.rg = a.r;
  f.pg0 = a.p0;
  f.pg1 = a.p1;
  f.partials = a.partials;
  f.bar = a.bar;
  f.ctl = a.ctl;
  f.tol = tol;
  f.maxit = maxit;
  f.spin_cycles = fc.spin_cycles;
  f.expected = (unsigned)G + (unsigned)std::max(0, fc.missing);
  f.guard = a.guard;
  *used = true;
  if ((e = cudaMemsetAsync(a.bar, 0, sizeof(FusedBar), a.st)) != cudaSuccess) {
    if (err) *err = std::string("resident CG barrier reset: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  void* args[] = {&f};
  {
    ProfScope ps(a.prof, KI_CG_RESIDENT, a.st);
    e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(kResThreads), args, pl.smem, a.st);
  }
  if (e != cudaSuccess) {
    if (err) *err = std::string("resident CG launch: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  if ((e = cudaMemcpyAsync(a.ctl_host, a.ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, a.st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(a.st)) != cudaSuccess) {
    if (err) *err = std::string("resident CG: ") + cudaGetErrorString(e);
    return LES_ERR_CUDA;
  }
  const SolverCtl& c = *a.ctl_host;
  if (iters) *iters = c.iter;
  if (rel) *rel = c.rel;
  // algorithmic traffic of the same CG written as streaming passes (as for
  // the streaming solver), so that the two report comparable rates
  if (a.prof) a.prof->bytes[KI_CG_RESIDENT] += (7.0 + 10.0 * c.iter) * (double)f.n * sizeof(T);
  switch (c.done) {
    case 1:
    case 4: return LES_OK;
    case 2: return LES_ERR_NOT_CONVERGED;
    case 3:
      if (err) *err = "poisson: breakdown (zero or non-finite p.Ap / residual)";
      return LES_ERR_NONFINITE;
    case 5:
      if (err) *err = "poisson: a grid barrier wait timed out";
      return LES_ERR_TIMEOUT;
    default:
      if (err) *err = "poisson: resident solver returned no status";
      return LES_ERR_CUDA;
  }
}

template int poisson_solve_resident<float>(const SolverArgs<float>&, const FusedCfg&, const float*, float*, double,
                                           int, int*, double*, std::string*, bool*);
template int poisson_solve_resident<double>(const SolverArgs<double>&, const FusedCfg&, const double*, double*,
                                            double, int, int*, double*, std::string*, bool*);

}  // namespace les
