// C ABI of the relativistic LBM library (declared in include/rlbm.h).
//
// Host side only: argument checks, workspace layout, constants, and the
// sequence of kernel launches on the caller's stream.  All arithmetic of the
// method runs in the kernel modules (kernels_*.cu).
#include "rlbm.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ops.h"

namespace rlbm {
namespace {

thread_local std::string g_create_error;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr int kStagePlanes = 4;

struct SampleLayout {
  rlbm_sample desc;
  DevSample dev;
  size_t buf_off[2];     // byte offsets of the two population buffers
  size_t buf_bytes;
  long long sites;
  double ghost[kMaxContacts][kQ];   // contact deviations f^eq - w
};

struct Quad {
  bool ok = false;
  double w1[4], w2[4], p0[4];
};

const Quad& quad() {
  static Quad q = [] {
    Quad r;
    r.ok = refine_quadrature(r.w1, r.w2, r.p0);
    return r;
  }();
  return q;
}

const PrecOps* ops_for(rlbm_prec p) {
  switch (p) {
    case RLBM_F64: return ops_f64();
    case RLBM_F32: return ops_f32();
    case RLBM_F16DEV: return ops_f16();
    case RLBM_BF16DEV: return ops_bf16();
  }
  return nullptr;
}

// Scale of the 16-bit relative deviation g = s (f - w) / w.
double storage_scale(rlbm_prec p) {
  if (p == RLBM_F16DEV) return 1024.0;    // |g| < 64 keeps |(f - w)/w| < 1/16 in range
  if (p == RLBM_BF16DEV) return 1.0;
  return 1.0;
}

std::string check_sample(const rlbm_sample& s) {
  char b[256];
  if (s.nx < 2 * RLBM_HOP_RADIUS + 1 || s.ny < 2 * RLBM_HOP_RADIUS + 1) {
    snprintf(b, sizeof b, "sample dims %dx%d below the minimum 11x11", s.nx, s.ny);
    return b;
  }
  if ((long long)s.nx * s.ny > (1LL << 31)) return "sample has more than 2^31 sites";
  if (!(s.tau > 0.5) || !std::isfinite(s.tau)) return "tau must be > 0.5";
  if (!(std::fabs(s.Fx) < 1e-2) || !(std::fabs(s.Fy) < 1e-2)) return "|F| must be < 1e-2";
  if (s.ncontacts < 0 || s.ncontacts > RLBM_MAX_CONTACTS) return "ncontacts out of range";
  for (int k = 0; k < s.ncontacts; ++k) {
    const rlbm_contact& c = s.contacts[k];
    if (c.edge < 0 || c.edge > 3) return "contact edge must be 0..3";
    if ((c.edge < 2 && s.periodic_y) || (c.edge >= 2 && s.periodic_x))
      return "contact on a periodic edge";
    const int len = c.edge < 2 ? s.nx : s.ny;
    if (c.length <= 0 || c.x0 < 0 || c.x0 + c.length > len) return "contact span off the edge";
    if (!(std::fabs(c.u_n) < 0.5) || !(c.n > 0) || !(c.T > 0)) return "contact state out of range";
  }
  return "";
}

}  // namespace

// Message for rlbm_last_error(NULL) from entry points without a context.
void set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }

}  // namespace rlbm

using namespace rlbm;

struct rlbm_ctx {
  rlbm_prec prec;
  const PrecOps* ops;
  cudaStream_t stream;
  int device;
  bool owns_workspace;
  unsigned char* ws;
  size_t ws_bytes;
  std::vector<SampleLayout> samples;
  std::vector<char> sample_ready;
  int cur;                    // which of the two buffers holds the current state
  bool initialised;
  long long steps;
  long long launches;
  size_t uprev_off, acc_off, err_off, ghost_off, stage_off;
  long long total_sites, max_sites;
  double* host_pinned;        // 2 doubles + error word staging
  std::string err;
};

namespace {

int fail(rlbm_ctx* c, int code, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b, sizeof b, fmt, ap);
  va_end(ap);
  if (c) c->err = b; else g_create_error = b;
  return code;
}

int cuda_fail(rlbm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, RLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Computes the layout of cfg; fills `out` when non-null.  Returns total bytes.
size_t plan(const rlbm_config* cfg, const PrecOps* ops, rlbm_ctx* out) {
  size_t off = 0;
  long long total = 0, maxs = 0;
  std::vector<SampleLayout> L(cfg->nsamples);
  for (int i = 0; i < cfg->nsamples; ++i) {
    const rlbm_sample& s = cfg->samples[i];
    SampleLayout& l = L[i];
    std::memset(&l, 0, sizeof l);
    l.desc = s;
    const int ldx = (int)align_up((size_t)s.nx, 32);
    const long long plane = (long long)align_up((size_t)ldx * s.ny, 64);
    l.buf_bytes = align_up((size_t)plane * kQ * ops->elem_bytes, 256);
    l.buf_off[0] = off;
    l.buf_off[1] = off + l.buf_bytes;
    off += 2 * l.buf_bytes;
    l.sites = (long long)s.nx * s.ny;
    DevSample& d = l.dev;
    d.nx = s.nx; d.ny = s.ny; d.ldx = ldx;
    d.periodic_x = s.periodic_x ? 1 : 0;
    d.periodic_y = s.periodic_y ? 1 : 0;
    d.ncontacts = s.ncontacts;
    d.plane = plane;
    d.site0 = total;
    d.inv_tau = 1.0 / s.tau;
    d.Fx = s.Fx; d.Fy = s.Fy;
    for (int k = 0; k < s.ncontacts; ++k) {
      d.cedge[k] = s.contacts[k].edge;
      d.clo[k] = s.contacts[k].x0;
      d.chi[k] = s.contacts[k].x0 + s.contacts[k].length;
    }
    total += l.sites;
    if (l.sites > maxs) maxs = l.sites;
  }
  const size_t uprev_off = off;
  off = align_up(off + (size_t)total * 2 * ops->real_bytes, 256);
  const size_t acc_off = off;
  off += 256;
  const size_t err_off = off;
  off += 256;
  const size_t ghost_off = off;
  off = align_up(off + (size_t)cfg->nsamples * kMaxContacts * kQ * sizeof(double), 256);
  const size_t stage_off = off;
  // FP64 staging: four planes of the largest sample (fields, or a chunk of
  // the state), and the 11x11 contact patch
  const size_t stage_doubles = std::max<size_t>((size_t)maxs * kStagePlanes, (size_t)(kQ + 4) * 121);
  off = align_up(off + stage_doubles * sizeof(double), 256);
  if (out) {
    out->samples = std::move(L);
    out->uprev_off = uprev_off;
    out->acc_off = acc_off;
    out->err_off = err_off;
    out->ghost_off = ghost_off;
    out->stage_off = stage_off;
    out->total_sites = total;
    out->max_sites = maxs;
  }
  return off;
}

int check_config(const rlbm_config* cfg, rlbm_ctx* c) {
  if (!cfg) return fail(c, RLBM_EINVAL, "config is NULL");
  if (!ops_for(cfg->prec)) return fail(c, RLBM_EINVAL, "unknown precision %d", (int)cfg->prec);
  if (cfg->nsamples < 1 || !cfg->samples) return fail(c, RLBM_EINVAL, "need nsamples >= 1");
  for (int i = 0; i < cfg->nsamples; ++i) {
    std::string e = check_sample(cfg->samples[i]);
    if (!e.empty()) return fail(c, RLBM_EINVAL, "sample %d: %s", i, e.c_str());
  }
  return RLBM_OK;
}

template <typename T>
T* at(rlbm_ctx* c, size_t off) { return reinterpret_cast<T*>(c->ws + off); }

void* buf(rlbm_ctx* c, int sample, int which) {
  return c->ws + c->samples[sample].buf_off[which];
}

// Ghost deviations f^eq(n_c, u_n * inward normal, T_c) - w of every contact
// (Sec. 3: contact sites do not evolve), formed once by the FP64 init kernel
// on a uniform 11 x 11 patch in the staging area.
int upload_ghosts(rlbm_ctx* c) {
  const int kP = 2 * RLBM_HOP_RADIUS + 1;
  std::vector<double> ghost((size_t)c->samples.size() * kMaxContacts * kQ, 0.0);
  double* stage = at<double>(c, c->stage_off);
  unsigned* err = at<unsigned>(c, c->err_off);
  for (size_t i = 0; i < c->samples.size(); ++i) {
    const rlbm_sample& s = c->samples[i].desc;
    for (int k = 0; k < s.ncontacts; ++k) {
      const rlbm_contact& ct = s.contacts[k];
      const double nx_ = ct.edge == 2 ? 1.0 : ct.edge == 3 ? -1.0 : 0.0;
      const double ny_ = ct.edge == 0 ? 1.0 : ct.edge == 1 ? -1.0 : 0.0;
      const double vals[4] = {ct.n, ct.u_n * nx_, ct.u_n * ny_, ct.T};
      // fields: 4 planes of kP*kP doubles after the 48*kP*kP population patch
      double* fields = stage + (size_t)kQ * kP * kP;
      std::vector<double> h((size_t)4 * kP * kP);
      for (int f = 0; f < 4; ++f)
        for (int s2 = 0; s2 < kP * kP; ++s2) h[(size_t)f * kP * kP + s2] = vals[f];
      cudaError_t e = cudaMemcpyAsync(fields, h.data(), h.size() * sizeof(double),
                                      cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "ghost upload");
      DevSample d{};
      d.nx = kP; d.ny = kP; d.ldx = kP; d.plane = (long long)kP * kP;
      // FP64 module regardless of the context precision: ghost values are FP64
      e = ops_f64()->init(stage, d, fields, fields + kP * kP, fields + 2 * kP * kP,
                          fields + 3 * kP * kP, err, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "ghost init kernel");
      c->launches++;
      std::vector<double> patch((size_t)kQ * kP * kP);
      e = cudaMemcpyAsync(patch.data(), stage, patch.size() * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "ghost readback");
      for (int q = 0; q < kQ; ++q) {
        // site 0 of direction plane q / 4, shell q % 4 (four shells per site vector)
        const double v = patch[(size_t)(q >> 2) * kP * kP * 4 + (q & 3)];
        c->samples[i].ghost[k][q] = v;
        ghost[(i * kMaxContacts + k) * kQ + q] = v;
      }
    }
  }
  // Device copy in the arithmetic type of the context.
  if (c->ops->real_bytes == sizeof(double)) {
    cudaError_t e = cudaMemcpyAsync(at<double>(c, c->ghost_off), ghost.data(),
                                    ghost.size() * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ghost copy");
  } else {
    std::vector<float> gf(ghost.size());
    for (size_t i = 0; i < ghost.size(); ++i) gf[i] = (float)ghost[i];
    cudaError_t e = cudaMemcpyAsync(at<float>(c, c->ghost_off), gf.data(),
                                    gf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ghost copy");
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ghost sync");
  return RLBM_OK;
}

const void* ghost_ptr(rlbm_ctx* c, int sample) {
  return c->ws + c->ghost_off + (size_t)sample * kMaxContacts * kQ * c->ops->real_bytes;
}

int check_sample_index(rlbm_ctx* c, int sample) {
  if (!c) return RLBM_EINVAL;
  if (sample < 0 || sample >= (int)c->samples.size())
    return fail(c, RLBM_EINVAL, "sample %d out of range", sample);
  return RLBM_OK;
}

}  // namespace

extern "C" {

int rlbm_version(void) { return 1; }

int rlbm_quadrature(double w1[4], double w2[4], double p0[4]) {
  const Quad& q = quad();
  if (!q.ok) return fail(nullptr, RLBM_EINVAL, "quadrature refinement did not converge");
  for (int j = 0; j < 4; ++j) { w1[j] = q.w1[j]; w2[j] = q.w2[j]; p0[j] = q.p0[j]; }
  return RLBM_OK;
}

int rlbm_workspace_size(const rlbm_config* cfg, size_t* bytes) {
  int r = check_config(cfg, nullptr);
  if (r) return r;
  if (!bytes) return fail(nullptr, RLBM_EINVAL, "bytes is NULL");
  *bytes = plan(cfg, ops_for(cfg->prec), nullptr);
  return RLBM_OK;
}

int rlbm_create(const rlbm_config* cfg, rlbm_ctx** out) {
  if (!out) return fail(nullptr, RLBM_EINVAL, "out is NULL");
  *out = nullptr;
  int r = check_config(cfg, nullptr);
  if (r) return r;
  const Quad& q = quad();
  if (!q.ok) return fail(nullptr, RLBM_EINVAL, "quadrature refinement did not converge");
  rlbm_ctx* c = new (std::nothrow) rlbm_ctx();
  if (!c) return fail(nullptr, RLBM_ENOMEM, "host allocation failed");
  c->prec = cfg->prec;
  c->ops = ops_for(cfg->prec);
  c->stream = static_cast<cudaStream_t>(cfg->stream);
  c->cur = 0;
  c->initialised = false;
  c->steps = 0;
  c->launches = 0;
  c->host_pinned = nullptr;
  cudaGetDevice(&c->device);
  const size_t need = plan(cfg, c->ops, c);
  c->sample_ready.assign(c->samples.size(), 0);
  if (cfg->workspace) {
    if (cfg->workspace_bytes < need || (reinterpret_cast<uintptr_t>(cfg->workspace) & 255)) {
      delete c;
      return fail(nullptr, RLBM_ENOMEM, "workspace too small or misaligned: need %zu bytes",
                  need);
    }
    c->ws = static_cast<unsigned char*>(cfg->workspace);
    c->owns_workspace = false;
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, RLBM_ENOMEM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
    }
    c->ws = static_cast<unsigned char*>(p);
    c->owns_workspace = true;
  }
  c->ws_bytes = need;
  cudaError_t e = cudaMallocHost((void**)&c->host_pinned, 256);
  if (e != cudaSuccess) { rlbm_destroy(c); return fail(nullptr, RLBM_ENOMEM, "pinned staging"); }
  const double w[2][4] = {{q.w1[0], q.w1[1], q.w1[2], q.w1[3]}, {q.w2[0], q.w2[1], q.w2[2], q.w2[3]}};
  e = c->ops->upload(q.p0, w, storage_scale(c->prec));
  if (e == cudaSuccess && c->ops != ops_f64()) e = ops_f64()->upload(q.p0, w, 1.0);
  if (e != cudaSuccess) { rlbm_destroy(c); return fail(nullptr, RLBM_ECUDA, "constant upload: %s", cudaGetErrorString(e)); }
  e = cudaMemsetAsync(c->ws + c->err_off, 0, 256, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + c->ghost_off, 0, c->stage_off - c->ghost_off, c->stream);
  if (e != cudaSuccess) { rlbm_destroy(c); return fail(nullptr, RLBM_ECUDA, "memset: %s", cudaGetErrorString(e)); }
  r = upload_ghosts(c);
  if (r) { std::string m = c->err; rlbm_destroy(c); return fail(nullptr, r, "%s", m.c_str()); }
  *out = c;
  return RLBM_OK;
}

void rlbm_destroy(rlbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  if (c->owns_workspace && c->ws) cudaFree(c->ws);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  delete c;
}

const char* rlbm_last_error(const rlbm_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

long long rlbm_steps_done(const rlbm_ctx* c) { return c ? c->steps : -1; }
long long rlbm_launch_count(const rlbm_ctx* c) { return c ? c->launches : -1; }

int rlbm_init(rlbm_ctx* c, int sample, const double* n, const double* ux, const double* uy,
              const double* T, int device_ptrs) {
  int r = check_sample_index(c, sample);
  if (r) return r;
  const int nnull = !n + !ux + !uy + !T;
  if (nnull != 0 && nnull != 4) return fail(c, RLBM_EINVAL, "give all four fields or none");
  SampleLayout& L = c->samples[sample];
  void* dst = buf(c, sample, c->cur);
  cudaError_t e;
  if (nnull == 4) {
    e = cudaMemsetAsync(dst, 0, L.buf_bytes, c->stream);   // rest state: f = w, delta = 0
    if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  } else {
    const double* fp[4] = {n, ux, uy, T};
    const double* dp[4];
    double* stage = at<double>(c, c->stage_off);
    for (int f = 0; f < 4; ++f) {
      if (device_ptrs) { dp[f] = fp[f]; continue; }
      double* d = stage + (size_t)f * L.sites;
      e = cudaMemcpyAsync(d, fp[f], (size_t)L.sites * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "field upload");
      dp[f] = d;
    }
    e = c->ops->init(dst, L.dev, dp[0], dp[1], dp[2], dp[3], at<unsigned>(c, c->err_off),
                     c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    c->launches++;
  }
  c->sample_ready[sample] = 1;
  c->initialised = std::all_of(c->sample_ready.begin(), c->sample_ready.end(),
                               [](char v) { return v != 0; });
  c->steps = 0;
  return RLBM_OK;
}

int rlbm_step(rlbm_ctx* c, int nsteps, double* residual) {
  if (!c) return RLBM_EINVAL;
  if (nsteps < 0) return fail(c, RLBM_EINVAL, "nsteps < 0");
  if (!c->initialised) return fail(c, RLBM_ESTATE, "rlbm_init or rlbm_set_state first");
  if (residual && nsteps < 2) return fail(c, RLBM_EINVAL, "residual needs nsteps >= 2");
  double* acc = at<double>(c, c->acc_off);
  unsigned* err = at<unsigned>(c, c->err_off);
  void* uprev = c->ws + c->uprev_off;
  if (residual) {
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  }
  for (int t = 0; t < nsteps; ++t) {
    int res = 0;
    if (residual && t == nsteps - 2) res = 1;
    if (residual && t == nsteps - 1) res = 2;
    for (size_t i = 0; i < c->samples.size(); ++i) {
      SampleLayout& L = c->samples[i];
      const bool force = L.desc.Fx != 0.0 || L.desc.Fy != 0.0;
      cudaError_t e = c->ops->step(buf(c, (int)i, c->cur), buf(c, (int)i, c->cur ^ 1), L.dev,
                                   ghost_ptr(c, (int)i), force, res, uprev, acc, err, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
      c->launches++;
    }
    c->cur ^= 1;
    c->steps++;
  }
  if (residual) {
    cudaError_t e = cudaMemcpyAsync(c->host_pinned, acc, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->host_pinned + 2, err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "residual readback");
    const double num = c->host_pinned[0], den = c->host_pinned[1];
    *residual = den > 0 ? std::sqrt(num / den) : (num == 0 ? 0.0 : INFINITY);
    unsigned bits;
    std::memcpy(&bits, c->host_pinned + 2, sizeof bits);
    if (bits) {
      cudaMemsetAsync(err, 0, sizeof(unsigned), c->stream);
      return fail(c, RLBM_ENAN, "device error word 0x%x (1 non-finite, 2 unphysical, 4 no convergence)", bits);
    }
  }
  return RLBM_OK;
}

int rlbm_check(rlbm_ctx* c) {
  if (!c) return RLBM_EINVAL;
  unsigned* err = at<unsigned>(c, c->err_off);
  cudaError_t e = cudaMemcpyAsync(c->host_pinned, err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "error word readback");
  unsigned bits;
  std::memcpy(&bits, c->host_pinned, sizeof bits);
  if (bits) {
    cudaMemsetAsync(err, 0, sizeof(unsigned), c->stream);
    return fail(c, RLBM_ENAN, "device error word 0x%x (1 non-finite, 2 unphysical, 4 no convergence)", bits);
  }
  return RLBM_OK;
}

int rlbm_moments(rlbm_ctx* c, int sample, double* n, double* ux, double* uy, double* T,
                 int device_ptrs) {
  int r = check_sample_index(c, sample);
  if (r) return r;
  if (!c->initialised) return fail(c, RLBM_ESTATE, "rlbm_init or rlbm_set_state first");
  SampleLayout& L = c->samples[sample];
  double* outp[4] = {n, ux, uy, T};
  double* dp[4];
  double* stage = at<double>(c, c->stage_off);
  for (int f = 0; f < 4; ++f)
    dp[f] = !outp[f] ? nullptr : device_ptrs ? outp[f] : stage + (size_t)f * L.sites;
  cudaError_t e = c->ops->moments(buf(c, sample, c->cur), L.dev, ghost_ptr(c, sample), dp[0],
                                  dp[1], dp[2], dp[3], at<unsigned>(c, c->err_off), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
  c->launches++;
  if (!device_ptrs) {
    for (int f = 0; f < 4; ++f) {
      if (!outp[f]) continue;
      e = cudaMemcpyAsync(outp[f], dp[f], (size_t)L.sites * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "field readback");
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  }
  return RLBM_OK;
}

int rlbm_get_state(rlbm_ctx* c, int sample, double* delta, int device_ptrs) {
  int r = check_sample_index(c, sample);
  if (r) return r;
  if (!delta) return fail(c, RLBM_EINVAL, "delta is NULL");
  SampleLayout& L = c->samples[sample];
  if (device_ptrs) {
    cudaError_t e = c->ops->get_state(buf(c, sample, c->cur), L.dev, 0, kQ, delta, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state kernel");
    c->launches++;
    return RLBM_OK;
  }
  double* st = at<double>(c, c->stage_off);
  for (int q0 = 0; q0 < kQ; q0 += kStagePlanes) {
    cudaError_t e = c->ops->get_state(buf(c, sample, c->cur), L.dev, q0, kStagePlanes, st, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state kernel");
    c->launches++;
    e = cudaMemcpyAsync(delta + (size_t)q0 * L.sites, st,
                        (size_t)L.sites * kStagePlanes * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "state readback");
  }
  return RLBM_OK;
}

int rlbm_set_state(rlbm_ctx* c, int sample, const double* delta, int device_ptrs) {
  int r = check_sample_index(c, sample);
  if (r) return r;
  if (!delta) return fail(c, RLBM_EINVAL, "delta is NULL");
  SampleLayout& L = c->samples[sample];
  if (device_ptrs) {
    cudaError_t e = c->ops->set_state(buf(c, sample, c->cur), L.dev, 0, kQ, delta, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state kernel");
    c->launches++;
  } else {
    double* st = at<double>(c, c->stage_off);
    for (int q0 = 0; q0 < kQ; q0 += kStagePlanes) {
      cudaError_t e = cudaMemcpyAsync(st, delta + (size_t)q0 * L.sites,
                                      (size_t)L.sites * kStagePlanes * sizeof(double),
                                      cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "state upload");
      e = c->ops->set_state(buf(c, sample, c->cur), L.dev, q0, kStagePlanes, st, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "set_state kernel");
      c->launches++;
      e = cudaStreamSynchronize(c->stream);   // staging is reused by the next chunk
      if (e != cudaSuccess) return cuda_fail(c, e, "sync");
    }
  }
  c->sample_ready[sample] = 1;
  c->initialised = std::all_of(c->sample_ready.begin(), c->sample_ready.end(),
                               [](char v) { return v != 0; });
  c->steps = 0;
  return RLBM_OK;
}

}  // extern "C"
