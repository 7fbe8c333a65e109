// les_dd.cu -- the pressure-correction Poisson solve (Sec. 2.4, compact
// operator of Appendix A) on one sub-domain of an x-y domain decomposition,
// the parallelisation the paper runs on TPU cores (Sec. 2.5; Sec. 4.2).
//
// A global nx x ny x nz grid (periodic in x and y; periodic in z or bounded by
// walls) is cut into px x py sub-domains of (nx / px) x (ny / py) x nz nodes,
// one per rank.  Each rank keeps its CG vectors with a one-node halo in x and
// y (the compact Laplacian reaches one node); before every matvec the four
// face strips of p are packed, exchanged with the four neighbours through a
// caller-supplied function (NCCL send / receive, peer copies, ...), and
// unpacked into the halo.  The iteration is the standard CG; the four dot
// products of an iteration (p.q, r.r, r.q, q.q, FP64 over the sub-domain)
// are summed over ranks by one caller-supplied all-reduce, and r'.r' =
// r.r - 2 alpha r.q + alpha^2 q.q gives beta without a second reduction.
//
// The decomposed step keeps a sub-domain's fields in a handle widened by
// LES_DD_HALO nodes on each side in x and y; this file also packs and unpacks
// those fields' halos (two exchanges: x strips over the owned rows, then y
// strips over the whole widened width, which carries the corners).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "les_internal.h"

struct les_dd {
  les_config cfg{};     // the global configuration
  int px = 1, py = 1, rx = 0, ry = 0;
  int nx = 0, ny = 0, nz = 0;  // local interior
  int x0 = 0, y0 = 0;          // global offset of the local interior
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  // padded vectors (nx + 2) x (ny + 2) x nz: x, r, p, q; face buffers
  void *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  void *send[4] = {}, *recv[4] = {};
  size_t face_bytes[4] = {};
  // strips of the decomposed step's field halos (LES_DD_HALO deep, up to
  // LES_DD_MAX_FIELDS fields), fcap bytes each
  void *fsend[4] = {}, *frecv[4] = {};
  size_t fcap = 0;
  double* partials = nullptr;  // [4][nblk]
  double* sums = nullptr;      // [4]
  double host[4] = {};         // host copy of the sums
  int nblk = 0;
  std::string err;
};

namespace {

using les::Grid;

struct DdGeom {
  int nx, ny, nz, walls;  // local interior
  long long pstride;      // (nx + 2) (ny + 2)
  int rowlen;             // nx + 2
  double idx2, idy2, idz2;
};

__host__ __device__ inline long long pidx(const DdGeom& g, int i, int j, int k) {
  return (long long)k * g.pstride + (long long)(j + 1) * g.rowlen + (i + 1);
}

// copy the caller's local array (node (i, j, k) at off + k sxy + j sx + i)
// into the padded interior, or back
template <typename T>
__global__ void k_dd_in(DdGeom g, les::DdLayout lay, const T* __restrict__ src, T* __restrict__ dst) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const int j = (int)((t / g.nx) % g.ny);
    const int k = (int)(t / ((long long)g.nx * g.ny));
    dst[pidx(g, i, j, k)] = src[lay.off + k * lay.sxy + (long long)j * lay.sx + i];
  }
}
template <typename T>
__global__ void k_dd_out(DdGeom g, les::DdLayout lay, const T* __restrict__ src, T* __restrict__ dst) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const int j = (int)((t / g.nx) % g.ny);
    const int k = (int)(t / ((long long)g.nx * g.ny));
    dst[lay.off + k * lay.sxy + (long long)j * lay.sx + i] = src[pidx(g, i, j, k)];
  }
}

// halos of the decomposed step's fields.  The widened sub-domain is
// nxe = nx + 2H by nye = ny + 2H by nz, owned nodes at [H, H + nx) x [H, H + ny).
// Phase 0 (x): the west strip is the owned columns H .. 2H-1, the east strip
// nx .. nx+H-1, over the owned rows; strip element ((f nz + k) ny + j) H + c.
// Phase 1 (y): the south strip is the rows H .. 2H-1, the north strip
// ny .. ny+H-1, over all nxe columns (the x halos filled in phase 0 carry
// the corners); element ((f nz + k) H + r) nxe + i.
struct FieldSet {
  void* f[LES_DD_MAX_FIELDS];
  int nf;
};
struct HaloGeom {
  int nx, ny, nz, nxe, nye;  // owned, widened
};
__host__ __device__ inline long long fidx(const HaloGeom& g, int i, int j, int k) {
  return ((long long)k * g.nye + j) * g.nxe + i;
}
template <typename T>
__global__ void k_dd_fpack(HaloGeom g, FieldSet fs, int phase, T* __restrict__ a, T* __restrict__ b) {
  constexpr int H = LES_DD_HALO;
  const int len = phase == 0 ? g.ny * H : g.nxe * H;  // one strip plane (per field and z)
  const long long n = (long long)fs.nf * g.nz * len;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t % len);
    const long long fk = t / len;
    const int k = (int)(fk % g.nz), f = (int)(fk / g.nz);
    const T* v = (const T*)fs.f[f];
    if (phase == 0) {
      const int j = H + e / H, c = e % H;
      a[t] = v[fidx(g, H + c, j, k)];
      b[t] = v[fidx(g, g.nx + c, j, k)];
    } else {
      const int r = e / g.nxe, i = e % g.nxe;
      a[t] = v[fidx(g, i, H + r, k)];
      b[t] = v[fidx(g, i, g.ny + r, k)];
    }
  }
}
// a: from the west (south) neighbour, its east (north) strip, into the halo
// below the owned range; b: from the east (north), into the halo above
template <typename T>
__global__ void k_dd_funpack(HaloGeom g, FieldSet fs, int phase, const T* __restrict__ a, const T* __restrict__ b) {
  constexpr int H = LES_DD_HALO;
  const int len = phase == 0 ? g.ny * H : g.nxe * H;
  const long long n = (long long)fs.nf * g.nz * len;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t % len);
    const long long fk = t / len;
    const int k = (int)(fk % g.nz), f = (int)(fk / g.nz);
    T* v = (T*)fs.f[f];
    if (phase == 0) {
      const int j = H + e / H, c = e % H;
      v[fidx(g, c, j, k)] = a[t];
      v[fidx(g, g.nx + H + c, j, k)] = b[t];
    } else {
      const int r = e / g.nxe, i = e % g.nxe;
      v[fidx(g, i, r, k)] = a[t];
      v[fidx(g, i, g.ny + H + r, k)] = b[t];
    }
  }
}

// face f of the interior into a contiguous strip: 0 west (i = 0), 1 east
// (i = nx-1), 2 south (j = 0), 3 north (j = ny-1); strips run over (j, k) or
// (i, k), first index fastest
template <typename T>
__global__ void k_dd_pack(DdGeom g, const T* __restrict__ v, T* w, T* e, T* s, T* n) {
  const long long nxz = (long long)g.ny * g.nz, nyz = (long long)g.nx * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * nxz + 2 * nyz;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < 2 * nxz) {
      const long long u = t < nxz ? t : t - nxz;
      const int j = (int)(u % g.ny), k = (int)(u / g.ny);
      if (t < nxz) w[u] = v[pidx(g, 0, j, k)];
      else e[u] = v[pidx(g, g.nx - 1, j, k)];
    } else {
      const long long t2 = t - 2 * nxz;
      const long long u = t2 < nyz ? t2 : t2 - nyz;
      const int i = (int)(u % g.nx), k = (int)(u / g.nx);
      if (t2 < nyz) s[u] = v[pidx(g, i, 0, k)];
      else n[u] = v[pidx(g, i, g.ny - 1, k)];
    }
  }
}
// the received strips into the halo: from the west neighbour (its east
// face) to i = -1, from the east to i = nx, south to j = -1, north to j = ny
template <typename T>
__global__ void k_dd_unpack(DdGeom g, T* v, const T* w, const T* e, const T* s, const T* n) {
  const long long nxz = (long long)g.ny * g.nz, nyz = (long long)g.nx * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * nxz + 2 * nyz;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < 2 * nxz) {
      const long long u = t < nxz ? t : t - nxz;
      const int j = (int)(u % g.ny), k = (int)(u / g.ny);
      if (t < nxz) v[pidx(g, -1, j, k)] = w[u];
      else v[pidx(g, g.nx, j, k)] = e[u];
    } else {
      const long long t2 = t - 2 * nxz;
      const long long u = t2 < nyz ? t2 : t2 - nyz;
      const int i = (int)(u % g.nx), k = (int)(u / g.nx);
      if (t2 < nyz) v[pidx(g, i, -1, k)] = s[u];
      else v[pidx(g, i, g.ny, k)] = n[u];
    }
  }
}

template <typename T>
__device__ __forceinline__ T zval(const DdGeom& g, const T* v, int i, int j, int k) {
  if (k < 0) k = g.walls ? 0 : g.nz - 1;            // mirror ghost / wrap
  else if (k >= g.nz) k = g.walls ? g.nz - 1 : 0;
  return v[pidx(g, i, j, k)];
}

// q = L_c p on the interior (halo of p filled) and, per block, the partial
// sums of p.q, r.r, r.q, q.q in FP64
template <typename T>
__global__ void __launch_bounds__(256) k_dd_matvec(DdGeom g, const T* __restrict__ p, const T* __restrict__ r,
                                                   T* __restrict__ q, double* partials) {
  __shared__ double sh[32];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const int j = (int)((t / g.nx) % g.ny);
    const int k = (int)(t / ((long long)g.nx * g.ny));
    const long long m = pidx(g, i, j, k);
    const double c = (double)p[m];
    const double lx = ((double)p[m + 1] - 2.0 * c + (double)p[m - 1]) * g.idx2;
    const double ly = ((double)p[m + g.rowlen] - 2.0 * c + (double)p[m - g.rowlen]) * g.idy2;
    const double lz = ((double)zval(g, p, i, j, k + 1) - 2.0 * c + (double)zval(g, p, i, j, k - 1)) * g.idz2;
    const T qv = (T)(lx + ly + lz);
    q[m] = qv;
    const double rv = (double)r[m], qd = (double)qv;
    acc[0] += c * qd;
    acc[1] += rv * rv;
    acc[2] += rv * qd;
    acc[3] += qd * qd;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double s = les::block_reduce<false>(acc[v], sh);
    if (threadIdx.x == 0) partials[(size_t)v * gridDim.x + blockIdx.x] = s;
  }
}

// fold the block partials in a fixed order
__global__ void k_dd_fold(const double* partials, int nblk, int nv, double* sums) {
  __shared__ double sh[32];
  for (int v = 0; v < nv; ++v) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += partials[(size_t)v * nblk + b];
    const double s = les::block_reduce<false>(a, sh);
    if (threadIdx.x == 0) sums[v] = s;
    __syncthreads();
  }
}

// x += alpha p; r -= alpha q; p = r + beta p
template <typename T>
__global__ void k_dd_update(DdGeom g, T* x, T* r, T* p, const T* q, double alpha, double beta) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const int j = (int)((t / g.nx) % g.ny);
    const int k = (int)(t / ((long long)g.nx * g.ny));
    const long long m = pidx(g, i, j, k);
    const T pv = p[m];
    x[m] = (T)((double)x[m] + alpha * (double)pv);
    const T rv = (T)((double)r[m] - alpha * (double)q[m]);
    r[m] = rv;
    p[m] = (T)((double)rv + beta * (double)pv);
  }
}

// per-block partial sums of one vector's interior (nv = 1) or of a.b
template <typename T>
__global__ void __launch_bounds__(256) k_dd_sum(DdGeom g, const T* a, const T* b, double* partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const int j = (int)((t / g.nx) % g.ny);
    const int k = (int)(t / ((long long)g.nx * g.ny));
    const long long m = pidx(g, i, j, k);
    acc += b ? (double)a[m] * (double)b[m] : (double)a[m];
  }
  const double s = les::block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// v = a - shift (interior); optionally also w = v and z = 0
template <typename T>
__global__ void k_dd_shift(DdGeom g, T* v, double shift) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const int j = (int)((t / g.nx) % g.ny);
    const int k = (int)(t / ((long long)g.nx * g.ny));
    const long long m = pidx(g, i, j, k);
    v[m] = (T)((double)v[m] - shift);
  }
}
// r = b - q, p = r (interior)
template <typename T>
__global__ void k_dd_residual(DdGeom g, const T* b, const T* q, T* r, T* p) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const int j = (int)((t / g.nx) % g.ny);
    const int k = (int)(t / ((long long)g.nx * g.ny));
    const long long m = pidx(g, i, j, k);
    const T rv = (T)((double)b[m] - (double)q[m]);
    r[m] = rv;
    p[m] = rv;
  }
}

DdGeom geom(const les_dd* d) {
  DdGeom g;
  g.nx = d->nx, g.ny = d->ny, g.nz = d->nz;
  g.walls = d->cfg.bc_z == LES_BC_WALLS;
  g.rowlen = d->nx + 2;
  g.pstride = (long long)(d->nx + 2) * (d->ny + 2);
  g.idx2 = 1.0 / (d->cfg.dx * d->cfg.dx);
  g.idy2 = 1.0 / (d->cfg.dy * d->cfg.dy);
  g.idz2 = 1.0 / (d->cfg.dz * d->cfg.dz);
  return g;
}

size_t layout(les_dd* d, char* base, bool dry) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    off = (off + 255) / 256 * 256;
    void* p = dry ? nullptr : base + off;
    off += bytes;
    return p;
  };
  const size_t es = d->cfg.precision == 64 ? 8 : 4;
  const size_t padded = (size_t)(d->nx + 2) * (d->ny + 2) * d->nz * es;
  d->x = take(padded);
  d->r = take(padded);
  d->p = take(padded);
  d->q = take(padded);
  d->face_bytes[0] = d->face_bytes[1] = (size_t)d->ny * d->nz * es;
  d->face_bytes[2] = d->face_bytes[3] = (size_t)d->nx * d->nz * es;
  for (int f = 0; f < 4; ++f) d->send[f] = take(d->face_bytes[f]);
  for (int f = 0; f < 4; ++f) d->recv[f] = take(d->face_bytes[f]);
  const int H = LES_DD_HALO;
  d->fcap = (size_t)LES_DD_MAX_FIELDS * d->nz * H * std::max(d->ny, d->nx + 2 * H) * es;
  for (int f = 0; f < 4; ++f) d->fsend[f] = take(d->fcap);
  for (int f = 0; f < 4; ++f) d->frecv[f] = take(d->fcap);
  d->partials = (double*)take((size_t)4 * d->nblk * sizeof(double));
  d->sums = (double*)take(4 * sizeof(double));
  return off + 256;
}

int fail(les_dd* d, int rc, const std::string& m) {
  d->err = m;
  return rc;
}

template <typename T>
int solve(les_dd* d, const les_dd_ops* ops, const T* rhs, T* xout, const les::DdLayout& lay, double tol, int maxit,
          int* iters, double* rel) {
  const DdGeom g = geom(d);
  const int nb = d->nblk;
  cudaStream_t st = d->st;
  T *x = (T*)d->x, *r = (T*)d->r, *p = (T*)d->p, *q = (T*)d->q;
  cudaError_t e;
  auto ck = [&](const char* what) -> int {
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(d, LES_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return LES_OK;
  };
  // sum over ranks of nv FP64 values folded from the block partials
  auto reduce = [&](int nv, double* out) -> int {
    k_dd_fold<<<1, 256, 0, st>>>(d->partials, nb, nv, d->sums);
    if ((e = cudaMemcpyAsync(d->host, d->sums, nv * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return fail(d, LES_ERR_CUDA, std::string("reduction readback: ") + cudaGetErrorString(e));
    if (ops->allreduce(ops->ctx, d->host, nv) != 0) return fail(d, LES_ERR_CUDA, "all-reduce callback failed");
    for (int v = 0; v < nv; ++v) out[v] = d->host[v];
    return LES_OK;
  };
  auto halo = [&](T* v) -> int {
    k_dd_pack<T><<<nb, 256, 0, st>>>(g, v, (T*)d->send[0], (T*)d->send[1], (T*)d->send[2], (T*)d->send[3]);
    if (ck("pack") != LES_OK) return LES_ERR_CUDA;
    if (ops->exchange(ops->ctx, d->send, d->recv, d->face_bytes, st) != 0)
      return fail(d, LES_ERR_CUDA, "halo exchange callback failed");
    k_dd_unpack<T><<<nb, 256, 0, st>>>(g, v, (const T*)d->recv[0], (const T*)d->recv[1], (const T*)d->recv[2],
                                      (const T*)d->recv[3]);
    return ck("unpack");
  };
  const double ntot = (double)d->cfg.nx * d->cfg.ny * d->cfg.nz;
  // b (mean-free) lives in q until the first matvec; x from the caller
  k_dd_in<T><<<nb, 256, 0, st>>>(g, lay, rhs, q);
  k_dd_in<T><<<nb, 256, 0, st>>>(g, lay, xout, x);
  if (ck("copy in") != LES_OK) return LES_ERR_CUDA;
  double s1[4];
  k_dd_sum<T><<<nb, 256, 0, st>>>(g, q, (const T*)nullptr, d->partials);
  if (reduce(1, s1) != LES_OK) return LES_ERR_CUDA;
  k_dd_shift<T><<<nb, 256, 0, st>>>(g, q, s1[0] / ntot);
  k_dd_sum<T><<<nb, 256, 0, st>>>(g, q, q, d->partials);
  if (reduce(1, s1) != LES_OK) return LES_ERR_CUDA;
  const double bn = std::sqrt(s1[0]);
  int it = 0;
  double rr = 0.0, relres = 0.0;
  int rc = LES_OK;
  if (bn == 0.0) {
    cudaMemsetAsync(x, 0, (size_t)g.pstride * g.nz * (d->cfg.precision == 64 ? 8 : 4), st);
  } else {
    // r = b - A x, p = r: A x into p's slot via the matvec (r holds b)
    if ((e = cudaMemcpyAsync(r, q, (size_t)g.pstride * g.nz * sizeof(T), cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
      return fail(d, LES_ERR_CUDA, "copy");
    if (halo(x) != LES_OK) return LES_ERR_CUDA;
    k_dd_matvec<T><<<nb, 256, 0, st>>>(g, x, r, q, d->partials);
    k_dd_residual<T><<<nb, 256, 0, st>>>(g, r, q, r, p);
    k_dd_sum<T><<<nb, 256, 0, st>>>(g, r, r, d->partials);
    if (ck("set-up") != LES_OK) return LES_ERR_CUDA;
    if (reduce(1, s1) != LES_OK) return LES_ERR_CUDA;
    rr = s1[0];
    relres = std::sqrt(rr) / bn;
    while (relres > tol && it < maxit) {
      if (halo(p) != LES_OK) return LES_ERR_CUDA;
      k_dd_matvec<T><<<nb, 256, 0, st>>>(g, p, r, q, d->partials);
      if (ck("matvec") != LES_OK) return LES_ERR_CUDA;
      double sm[4];
      if (reduce(4, sm) != LES_OK) return LES_ERR_CUDA;
      if (!(sm[0] != 0.0) || !std::isfinite(sm[0]))
        return fail(d, LES_ERR_NONFINITE, "CG breakdown: p.Ap is zero or not finite");
      const double alpha = sm[1] / sm[0];
      double rr_new = sm[1] - 2.0 * alpha * sm[2] + alpha * alpha * sm[3];
      if (rr_new < 0.0) rr_new = 0.0;
      const double beta = rr_new / sm[1];
      k_dd_update<T><<<nb, 256, 0, st>>>(g, x, r, p, q, alpha, beta);
      if (ck("update") != LES_OK) return LES_ERR_CUDA;
      rr = rr_new;
      ++it;
      relres = std::sqrt(rr) / bn;
    }
    if (relres > tol) rc = LES_ERR_NOT_CONVERGED;
  }
  // gauge: zero mean
  k_dd_sum<T><<<nb, 256, 0, st>>>(g, x, (const T*)nullptr, d->partials);
  if (reduce(1, s1) != LES_OK) return LES_ERR_CUDA;
  k_dd_shift<T><<<nb, 256, 0, st>>>(g, x, s1[0] / ntot);
  k_dd_out<T><<<nb, 256, 0, st>>>(g, lay, x, xout);
  if (ck("copy out") != LES_OK) return LES_ERR_CUDA;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(d, LES_ERR_CUDA, cudaGetErrorString(e));
  if (iters) *iters = it;
  if (rel) *rel = relres;
  return rc;
}

}  // namespace

namespace les {

template <typename T>
int dd_solve(les_dd* d, const les_dd_ops* ops, const T* rhs, T* x, const DdLayout& lay, double tol, int maxit,
             int* iters, double* rel, std::string* err) {
  const int rc = solve<T>(d, ops, rhs, x, lay, tol, maxit, iters, rel);
  if (rc != LES_OK && rc != LES_ERR_NOT_CONVERGED && err) *err = d->err;
  return rc;
}
template int dd_solve<float>(les_dd*, const les_dd_ops*, const float*, float*, const DdLayout&, double, int, int*,
                             double*, std::string*);
template int dd_solve<double>(les_dd*, const les_dd_ops*, const double*, double*, const DdLayout&, double, int,
                              int*, double*, std::string*);

void dd_widened_shape(const les_dd* d, int* nxe, int* nye, int* nz) {
  *nxe = d->nx + 2 * LES_DD_HALO;
  *nye = d->ny + 2 * LES_DD_HALO;
  *nz = d->nz;
}

const les_config& dd_config(const les_dd* d) { return d->cfg; }

template <typename T>
static int halo_exchange_t(les_dd* d, const les_dd_ops* ops, void* const* fields, int nf, cudaStream_t st,
                           std::string* err) {
  constexpr int H = LES_DD_HALO;
  HaloGeom g{d->nx, d->ny, d->nz, d->nx + 2 * H, d->ny + 2 * H};
  FieldSet fs{};
  for (int f = 0; f < nf; ++f) fs.f[f] = fields[f];
  fs.nf = nf;
  for (int phase = 0; phase < 2; ++phase) {
    const long long len = phase == 0 ? (long long)g.ny * H : (long long)g.nxe * H;
    const long long n = (long long)nf * g.nz * len;
    const size_t b = (size_t)n * sizeof(T);
    const size_t sizes[4] = {phase == 0 ? b : 0, phase == 0 ? b : 0, phase == 1 ? b : 0, phase == 1 ? b : 0};
    const int lo = phase == 0 ? 0 : 2, hi = lo + 1;
    const unsigned nb = (unsigned)std::min<long long>((n + 255) / 256, 1024);
    k_dd_fpack<T><<<nb, 256, 0, st>>>(g, fs, phase, (T*)d->fsend[lo], (T*)d->fsend[hi]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      if (err) *err = std::string("halo pack: ") + cudaGetErrorString(e);
      return LES_ERR_CUDA;
    }
    if (ops->exchange(ops->ctx, d->fsend, d->frecv, sizes, st) != 0) {
      if (err) *err = "halo exchange callback failed";
      return LES_ERR_CUDA;
    }
    k_dd_funpack<T><<<nb, 256, 0, st>>>(g, fs, phase, (const T*)d->frecv[lo], (const T*)d->frecv[hi]);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      if (err) *err = std::string("halo unpack: ") + cudaGetErrorString(e);
      return LES_ERR_CUDA;
    }
  }
  return LES_OK;
}

int dd_halo_exchange(les_dd* d, const les_dd_ops* ops, void* const* fields, int nf, cudaStream_t st,
                     std::string* err) {
  if (nf < 1 || nf > LES_DD_MAX_FIELDS) return LES_ERR_INVALID_ARG;
  return d->cfg.precision == 64 ? halo_exchange_t<double>(d, ops, fields, nf, st, err)
                                : halo_exchange_t<float>(d, ops, fields, nf, st, err);
}

}  // namespace les

extern "C" {

int les_dd_workspace_bytes(const les_config* cfg, int32_t px, int32_t py, size_t* bytes) {
  if (!cfg || !bytes || cfg->struct_size != sizeof(les_config) || px < 1 || py < 1) return LES_ERR_INVALID_ARG;
  if (cfg->nx % px || cfg->ny % py || cfg->nz < 2 || (cfg->precision != 32 && cfg->precision != 64))
    return LES_ERR_INVALID_ARG;
  les_dd tmp;
  tmp.cfg = *cfg;
  tmp.nx = cfg->nx / px;
  tmp.ny = cfg->ny / py;
  tmp.nz = cfg->nz;
  tmp.nblk = 1024;
  *bytes = layout(&tmp, nullptr, true);
  return LES_OK;
}

int les_dd_create(const les_config* cfg, int32_t px, int32_t py, int32_t rx, int32_t ry, void* workspace,
                  size_t bytes, void* stream, les_dd** out) {
  if (!out) return LES_ERR_INVALID_ARG;
  *out = nullptr;
  size_t need = 0;
  if (les_dd_workspace_bytes(cfg, px, py, &need) != LES_OK || rx < 0 || rx >= px || ry < 0 || ry >= py ||
      !workspace || bytes < need || ((uintptr_t)workspace % 256) != 0)
    return LES_ERR_INVALID_ARG;
  if (cfg->poisson_op != LES_OP_COMPACT) return LES_ERR_INVALID_ARG;
  les_dd* d = new (std::nothrow) les_dd();
  if (!d) return LES_ERR_INVALID_ARG;
  d->cfg = *cfg;
  d->px = px, d->py = py, d->rx = rx, d->ry = ry;
  d->nx = cfg->nx / px, d->ny = cfg->ny / py, d->nz = cfg->nz;
  d->x0 = rx * d->nx, d->y0 = ry * d->ny;
  d->st = (cudaStream_t)stream;
  d->ws = (char*)workspace;
  d->ws_bytes = bytes;
  d->nblk = 1024;
  layout(d, d->ws, false);
  cudaError_t e = cudaMemsetAsync(d->ws, 0, need, d->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->st);
  if (e != cudaSuccess) {
    delete d;
    return LES_ERR_CUDA;
  }
  *out = d;
  return LES_OK;
}

void les_dd_destroy(les_dd* d) { delete d; }

int les_dd_local_shape(const les_dd* d, int32_t* nx, int32_t* ny, int32_t* nz, int32_t* x0, int32_t* y0) {
  if (!d) return LES_ERR_INVALID_ARG;
  if (nx) *nx = d->nx;
  if (ny) *ny = d->ny;
  if (nz) *nz = d->nz;
  if (x0) *x0 = d->x0;
  if (y0) *y0 = d->y0;
  return LES_OK;
}

int les_dd_poisson_solve(les_dd* d, const les_dd_ops* ops, const void* d_rhs, void* d_x, double rtol,
                         int32_t maxit, int32_t* iters, double* rel_res) {
  if (!d || !ops || !ops->exchange || !ops->allreduce || !d_rhs || !d_x || !(rtol > 0) || maxit < 0)
    return LES_ERR_INVALID_ARG;
  int it = 0;
  double rel = 0.0;
  const les::DdLayout lay{0, (long long)d->nx * d->ny, d->nx};  // contiguous local arrays
  const int rc = d->cfg.precision == 64
                     ? solve<double>(d, ops, (const double*)d_rhs, (double*)d_x, lay, rtol, maxit, &it, &rel)
                     : solve<float>(d, ops, (const float*)d_rhs, (float*)d_x, lay, rtol, maxit, &it, &rel);
  if (iters) *iters = it;
  if (rel_res) *rel_res = rel;
  return rc;
}

const char* les_dd_last_error(const les_dd* d) { return d ? d->err.c_str() : "no sub-domain"; }

}  // extern "C"
