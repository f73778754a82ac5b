// gm_lib.cu -- host side of libgm: argument checks, workspace layout, kernel
// launches and the LM iteration loop behind the C ABI of include/gm.h.
// The per-galaxy kernels of the headers are compiled here only (gm_inst_*.cu hold the tile kernels).
#define GM_HOST_TU 1
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <vector>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <set>

#include "../../include/gm.h"
#include "gm_adjoint.cuh"
#include "gm_fused.cuh"
#include "gm_geom.cuh"
#include "gm_instances.h"
#include "gm_lm.cuh"

namespace gm {
// the tile kernels are instantiated in gm_inst_*.cu
#define GM_X(M, P, C, W) extern template __global__ void k_fused<M, P, C, W>(const __grid_constant__ FusedArgs);
GM_FUSED_ALL(GM_X)
#undef GM_X
extern template __global__ void k_adjoint<ADJ_RESID>(const __grid_constant__ AdjArgs);
extern template __global__ void k_adjoint<ADJ_GRAD>(const __grid_constant__ AdjArgs);
#define GM_X(P) extern template __global__ void k_adj_resid<P>(const __grid_constant__ PixArgs);
GM_RESID_ALL(GM_X)
#undef GM_X
#define GM_X(P) extern template __global__ void k_adj_deriv<P>(const __grid_constant__ PixArgs);
GM_DERIV_ALL(GM_X)
#undef GM_X
}  // namespace gm

using namespace gm;

// Scratch of gm_chi2_grad_noalloc: a fixed array in device memory, reserved on
// every GPU that loads this library.  Host code must not use its name as a
// device address: the address comes from cudaGetSymbolAddress (see
// noalloc_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[GM_NOALLOC_SCRATCH_BYTES];

namespace {

thread_local char g_err[512] = "no error";
// gm_test_starve_next_pass: the poll limit of the next tile-kernel launch made by
// this thread whose first block is to skip its first window load (0: none armed).
thread_local unsigned g_starve_polls = 0;

// The armed starvation (once), or false.
bool take_starve(unsigned* polls) {
  if (!g_starve_polls) return false;
  *polls = g_starve_polls;
  g_starve_polls = 0;
  return true;
}
thread_local gm_fit_stats g_stats;
thread_local bool g_have_stats = false;
// CUDA events timing the passes of gm_fit_batch, created on first use and kept
// for the life of the thread (four per iteration: profile start, tile kernel
// start, tile kernel end, LM step end).
thread_local std::vector<cudaEvent_t> g_events;
// CUDA events around the kernel groups of gm_grad_adjoint (six boundaries), and
// whether the thread's last call recorded them.
thread_local cudaEvent_t g_adj_events[6] = {};
thread_local bool g_adj_timed = false;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define GM_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(GM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define GM_LAUNCHED(what)                                                                         \
  do {                                                                                            \
    cudaError_t e_ = cudaGetLastError();                                                          \
    if (e_ != cudaSuccess) return fail(GM_E_CUDA, "launch %s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kMaxP1 = 10;  // largest free-parameter count served by the one-pair-per-thread kernel

// Everything derived from the model description once per call.
struct Plan {
  DescDev dd;
  int conv[kMaxComp];
  int chan_of_slot[kMaxSlots];  // output channel of a free slot (1 + accumulator index), -1 fixed
  int Pc;                       // free slots touching a convolved component
  int nch_conv, ncp, nch_tot, nacc;
  int any_unconv;
  int comp_chan[kMaxComp];
};

// Parameter count of component c: the profile's, plus B when it is boxy.
int comp_np(const gm_model_desc* d, int c) {
  const int np = n_params(d->comp[c].kind);
  return np < 0 ? np : np + (d->has_box[c] ? 1 : 0);
}

int check_desc(const gm_model_desc* d) {
  if (!d) return fail(GM_E_INVAL, "desc is NULL");
  if (d->n_comp < 1 || d->n_comp > GM_MAX_COMP)
    return fail(GM_E_INVAL, "n_comp=%d outside 1..%d", d->n_comp, GM_MAX_COMP);
  if (d->n_slots < 1 || d->n_slots > GM_MAX_SLOTS)
    return fail(GM_E_INVAL, "n_slots=%d outside 1..%d", d->n_slots, GM_MAX_SLOTS);
  for (int c = 0; c < d->n_comp; ++c) {
    if (d->has_box[c]) {
      const int k = d->comp[c].kind;
      if (k != SERSIC && k != EXPDISK && k != GAUSSIAN && k != MOFFAT)
        return fail(GM_E_UNSUPPORTED, "component %d: boxiness is built for Sersic, exponential, Gaussian and Moffat", c);
    }
    const int np = comp_np(d, c);
    if (np < 0) return fail(GM_E_INVAL, "component %d has unknown kind %d", c, d->comp[c].kind);
    for (int k = 0; k < np; ++k)
      if (d->comp[c].slot[k] < 0 || d->comp[c].slot[k] >= d->n_slots)
        return fail(GM_E_INVAL, "component %d parameter %d uses slot %d outside 0..%d", c, k, d->comp[c].slot[k],
                    d->n_slots - 1);
  }
  int nfree = 0;
  for (int s = 0; s < d->n_slots; ++s) nfree += d->is_free[s] ? 1 : 0;
  if (nfree > GM_MAX_FREE) return fail(GM_E_INVAL, "%d free parameters exceed %d", nfree, GM_MAX_FREE);
  for (int s = 0; s < d->n_slots; ++s) {
    if (!(d->lo[s] <= d->hi[s])) return fail(GM_E_INVAL, "slot %d has lo > hi", s);
    if (d->is_log[s] && !(d->lo[s] > 0.0)) return fail(GM_E_INVAL, "log slot %d needs lo > 0", s);
  }
  for (int c = 0; c < d->n_comp; ++c) {
    if (!d->amp_is_mag[c]) continue;
    const int k = d->comp[c].kind;
    if (k == KING || k == SKY || k == TSKY)
      return fail(GM_E_UNSUPPORTED, "component %d: kind %d has no magnitude relation", c, k);
    if (d->is_log[d->comp[c].slot[4]])
      return fail(GM_E_INVAL, "component %d: a magnitude slot is fitted linearly (is_log must be 0)", c);
    if (!std::isfinite(d->mag_zero[c])) return fail(GM_E_INVAL, "component %d: mag_zero is not finite", c);
  }
  for (int c = 0; c < d->n_comp; ++c) {
    if (!d->has_box[c]) continue;
    const int bs = d->comp[c].slot[n_params(d->comp[c].kind)];
    if (!(d->lo[bs] > -2.0)) return fail(GM_E_INVAL, "component %d: the boxiness slot needs lo > -2", c);
    if (d->is_log[bs]) return fail(GM_E_INVAL, "component %d: the boxiness slot is fitted linearly", c);
  }
  return GM_OK;
}

int check_hwk(int H, int W, int K, const char* what, int g) {
  if (H < 1 || H > 4096 || W < 1 || W > 4096)
    return g < 0 ? fail(GM_E_INVAL, "%s stamp %dx%d outside 1..4096", what, H, W)
                 : fail(GM_E_INVAL, "%s stamp %d is %dx%d, outside 1..4096", what, g, H, W);
  if (K < 1 || K > 63 || (K % 2) == 0)
    return g < 0 ? fail(GM_E_INVAL, "%s PSF side K=%d must be odd, 1..63", what, K)
                 : fail(GM_E_INVAL, "%s PSF %d has side %d; it must be odd, 1..63", what, g, K);
  return GM_OK;
}

// Sizes only (what the workspace queries need).
int check_sizes(const gm_batch* b) {
  if (!b) return fail(GM_E_INVAL, "batch is NULL");
  if (b->n_gal < 0) return fail(GM_E_INVAL, "n_gal=%d < 0", b->n_gal);
  if (b->geom) return GM_OK;  // per-galaxy sizes are checked by plan_geom
  return check_hwk(b->H, b->W, b->K, "batch", -1);
}

int check_batch(const gm_batch* b, bool need_data) {
  int rc = check_sizes(b);
  if (rc) return rc;
  if (b->n_gal > 0) {
    if (!b->psf) return fail(GM_E_INVAL, "batch.psf is NULL");
    if (need_data && (!b->image || !b->sigma)) return fail(GM_E_INVAL, "batch.image/sigma is NULL");
  }
  return GM_OK;
}

// mode: MODE_MODEL (want_comp: per-component channels) or MODE_NORMAL
int make_plan(const gm_model_desc* d, int mode, bool want_comp, Plan* pl) {
  int rc = check_desc(d);
  if (rc) return rc;
  std::memset(pl, 0, sizeof(*pl));
  DescDev& D = pl->dd;
  D.n_comp = d->n_comp;
  D.n_slots = d->n_slots;
  bool touches_conv[kMaxSlots] = {};
  for (int c = 0; c < d->n_comp; ++c) {
    D.kind[c] = d->comp[c].kind;
    D.np[c] = comp_np(d, c);
    D.box[c] = d->has_box[c] ? 1 : 0;
    D.mag[c] = d->amp_is_mag[c] ? 1 : 0;
    D.mag_zero[c] = d->mag_zero[c];
    pl->conv[c] = d->comp[c].convolve ? 1 : 0;
    if (!pl->conv[c]) pl->any_unconv = 1;
    for (int k = 0; k < 8; ++k) D.slot[c][k] = k < D.np[c] ? d->comp[c].slot[k] : 0;
    if (pl->conv[c])
      for (int k = 0; k < D.np[c]; ++k) touches_conv[D.slot[c][k]] = true;
    if (!is_flat(D.kind[c])) D.is_pa[D.slot[c][3]] = 1;
  }
  for (int s = 0; s < d->n_slots; ++s) {
    D.is_log[s] = d->is_log[s] ? 1 : 0;
    D.lo[s] = d->lo[s];
    D.hi[s] = d->hi[s];
    pl->chan_of_slot[s] = -1;
  }
  // axis-ratio groups that may be rewritten from q > 1 to 1/q: every slot a
  // component of the group uses as axis ratio, position angle or scale length
  // must be used in that role only by components sharing the group's q slot
  auto role = [](int kind, int k) {
    if (is_flat(kind)) return 0;
    if (k == 2) return 1;
    if (k == 3) return 2;
    if (k == 5 || (kind == KING && k == 6)) return 3;
    return 0;
  };
  D.n_canon = 0;
  for (int c = 0; c < d->n_comp; ++c) {
    if (is_flat(D.kind[c])) continue;
    const int qs = D.slot[c][2];
    bool seen = false;
    for (int k = 0; k < D.n_canon; ++k) seen = seen || D.canon[k].q_slot == qs;
    if (seen) continue;
    bool ok = true;
    for (int c1 = 0; c1 < d->n_comp && ok; ++c1) {
      if (is_flat(D.kind[c1]) || D.slot[c1][2] != qs) continue;
      for (int k1 = 0; k1 < D.np[c1] && ok; ++k1) {
        const int r1 = role(D.kind[c1], k1);
        if (!r1) continue;
        for (int c2 = 0; c2 < d->n_comp; ++c2)
          for (int k2 = 0; k2 < D.np[c2]; ++k2)
            if (D.slot[c2][k2] == D.slot[c1][k1] &&
                (is_flat(D.kind[c2]) || D.slot[c2][2] != qs || role(D.kind[c2], k2) != r1))
              ok = false;
      }
    }
    if (!ok) continue;
    CanonGroup& cg = D.canon[D.n_canon++];
    cg.q_slot = qs;
    cg.n_pa = cg.n_scale = 0;
    for (int c1 = 0; c1 < d->n_comp; ++c1) {
      if (is_flat(D.kind[c1]) || D.slot[c1][2] != qs) continue;
      for (int k1 = 0; k1 < D.np[c1]; ++k1) {
        const int r1 = role(D.kind[c1], k1), s1 = D.slot[c1][k1];
        if (r1 == 2) {
          bool dup = false;
          for (int i = 0; i < cg.n_pa; ++i) dup = dup || cg.pa[i] == s1;
          if (!dup) cg.pa[cg.n_pa++] = s1;
        } else if (r1 == 3) {
          bool dup = false;
          for (int i = 0; i < cg.n_scale; ++i) dup = dup || cg.scale[i] == s1;
          if (!dup) cg.scale[cg.n_scale++] = s1;
        }
      }
    }
  }
  // accumulator order: free slots of convolved components first, then the rest
  int P = 0;
  for (int s = 0; s < d->n_slots; ++s)
    if (d->is_free[s] && touches_conv[s]) D.free_slot[P++] = s;
  pl->Pc = P;
  for (int s = 0; s < d->n_slots; ++s)
    if (d->is_free[s] && !touches_conv[s]) D.free_slot[P++] = s;
  D.P = P;
  for (int f = 0; f < P; ++f) pl->chan_of_slot[D.free_slot[f]] = 1 + f;
  for (int c = 0; c < kMaxComp; ++c) pl->comp_chan[c] = -1;
  if (mode == MODE_NORMAL) {
    pl->nch_conv = 1 + pl->Pc;
    pl->nch_tot = 1 + P;
    pl->nacc = 1 + P + P * (P + 1) / 2;
  } else {
    int nc = 1;
    if (want_comp)
      for (int c = 0; c < d->n_comp; ++c)
        if (pl->conv[c]) pl->comp_chan[c] = nc++;
    pl->nch_conv = nc;
    int nt = nc;
    if (want_comp)
      for (int c = 0; c < d->n_comp; ++c)
        if (!pl->conv[c]) pl->comp_chan[c] = nt++;
    pl->nch_tot = nt;
    pl->nacc = 0;
  }
  pl->ncp = (pl->nch_conv + 1) / 2;
  if (pl->ncp > kMaxPairs)
    return fail(GM_E_UNSUPPORTED, "%d correlated channels exceed %d", pl->nch_conv, 2 * kMaxPairs);
  return GM_OK;
}

// The per-launch model description both kernels read.
ChanMap chan_map(const Plan& pl) {
  ChanMap m;
  std::memset(&m, 0, sizeof(m));
  const DescDev& D = pl.dd;
  m.n_comp = D.n_comp;
  for (int c = 0; c < D.n_comp; ++c) {
    m.kind[c] = D.kind[c] | (D.mag[c] ? kMagFlag : 0) | (D.box[c] ? kBoxFlag : 0);
    m.conv[c] = pl.conv[c];
    m.np[c] = D.np[c];
    m.comp_chan[c] = pl.comp_chan[c];
    for (int k = 0; k < 8; ++k) {
      m.slot[c][k] = D.slot[c][k];
      m.chan[c][k] = (pl.nacc > 0 && k < D.np[c]) ? pl.chan_of_slot[D.slot[c][k]] : -1;
    }
  }
  m.any_unconv = pl.any_unconv;
  m.nch_conv = pl.nch_conv;
  m.ncp = pl.ncp;
  m.nch_tot = pl.nch_tot;
  m.n_slots = D.n_slots;
  // a lone unconvolved flat sky (no magnitude or boxiness flag) whose level, when free,
  // owns the last channel: the tile kernel and the adjoint's residuals apply it without
  // evaluating the component
  m.sky_comp = m.sky_ch = -1;
  int n_unconv = 0, last = -1;
  for (int c = 0; c < D.n_comp; ++c)
    if (!m.conv[c]) ++n_unconv, last = c;
  // one convolved component, every parameter free, d/dp_k on channel 1 + k
  m.ident_comp = -1;
  if (pl.nacc > 0 && D.n_comp - n_unconv == 1) {
    int cm = 0;
    while (!m.conv[cm]) ++cm;
    bool ident = m.nch_conv == 1 + m.np[cm] && m.np[cm] <= 8;
    for (int k = 0; k < m.np[cm]; ++k) ident = ident && m.chan[cm][k] == 1 + k;
    if (ident) m.ident_comp = cm;
  }
  if (n_unconv == 1 && m.kind[last] == SKY) {
    const int ch = m.chan[last][0];
    if (ch < 0 ? m.nch_tot == m.nch_conv : (ch == m.nch_tot - 1 && m.nch_tot == m.nch_conv + 1)) {
      m.sky_comp = last;
      m.sky_ch = ch;
    }
  }
  return m;
}

typedef void (*FusedKernel)(FusedArgs);

// A launch shape of two pairs per thread in four groups runs the 512-thread instance.
bool wide_shape(int cpt, int groups) { return cpt == 2 && groups > 2; }

// The fused kernel for (mode, P, pairs per thread, wide), or nullptr when not built.
FusedKernel pick_kernel(int mode, int P, int cpt, bool wide) {
#define GM_X(M, PP, C, W) \
  if (mode == M && (M == MODE_MODEL || P == PP) && cpt == C && (int)wide == W) return k_fused<M, PP, C, W>;
  GM_FUSED_ALL(GM_X)
#undef GM_X
  return nullptr;
}

// Launch shapes: pp pairs per pass, cpt pairs per thread, groups of 128 threads.  One
// pair per thread: up to 4 groups; two pairs per thread: up to 2 groups, or 4 groups
// with 4 pairs per pass (each two groups split two pairs by PSF rows) or with 2 (all
// four groups split both pairs).
bool shape_valid(int pp, int cpt, int groups) {
  if (pp < 1 || pp > kMaxPassPairs || (cpt != 1 && cpt != 2) || groups < 1) return false;
  if (cpt == 1) return groups <= 4 && pp <= groups;
  if (groups == 4) return pp == 4 || pp == 2;
  return groups <= 2 && pp <= 2 * groups;
}

struct Smem {
  int pp, cpt, groups, passes, plane, off_psf, off_in, off_out, off_cc, off_scale, off_red, off_bar, off_info, total,
      threads;
};

// Channel pairs per thread of the fused kernel by default: one (more warps) unless the
// reduction of many free parameters needs the register budget of 256 threads.
int pick_cpt(const Plan& pl) { return (pl.nacc == 0 || pl.dd.P <= kMaxP1) ? 1 : 2; }

// Shared-memory carve-up of one fused CTA for `pp` channel pairs per pass,
// `groups` groups of 128 threads holding up to `cpt` pairs each, and PSF sides
// up to K.  Each pair plane holds a (32+K-1) x window_pitch(K) window and
// starts at a 128-byte boundary (TMA destinations must be 128-byte aligned).
Smem smem_layout(const Plan& pl, int K, int n_comp, int n_slots, int pp, int cpt, int groups) {
  Smem s;
  s.pp = pp;
  s.cpt = cpt;
  s.groups = groups;
  s.passes = (pl.ncp + pp - 1) / pp;
  s.threads = kGroupThreads * groups;
  const int HH = kTile + K - 1;
  const size_t plane_bytes = ((size_t)HH * window_pitch(K) * 8 + 127) / 128 * 128;
  s.plane = (int)(plane_bytes / 8);
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    const size_t o = off;
    off += bytes;
    return (int)o;
  };
  s.off_in = take((size_t)pp * plane_bytes, 128);
  s.off_psf = take((size_t)K * psf_row_floats(K) * 4, 16);
  s.off_out = take((size_t)pl.nch_tot * kTilePix * 4, 16);
  s.off_cc = take((size_t)2 * n_comp * kCC * 4, 16);             // two items' constants
  s.off_scale = take((size_t)2 * scale_stride(n_slots) * 4, 16);
  s.off_red = take((size_t)(s.threads / 32) * std::max(pl.nacc, 1) * 4, 16);
  s.off_bar = take(16, 16);
  s.off_info = take(2 * sizeof(ItemInfo), 16);
  s.total = (int)off;
  return s;
}

// Launch shapes set by the autotuner (gm_tune_set), keyed by (largest PSF side, free parameters).
struct TuneShape {
  int pp, cpt, groups;
};
std::mutex g_tune_mu;
std::map<std::pair<int, int>, TuneShape> g_tune;
thread_local TuneShape g_last_shape = {0, 0, 0};

// A shape the fused kernel can run: its instance exists, every pair of a pass has a
// thread group (pp <= cpt * groups, the thread count within the instance's launch
// bound) and the carve-up fits the device.
bool shape_ok(const Plan& pl, int K, int n_comp, int n_slots, int smem_optin, int mode, const TuneShape& t,
              Smem* out) {
  if (!shape_valid(t.pp, t.cpt, t.groups) || t.pp > pl.ncp) return false;
  if (!pick_kernel(mode, pl.dd.P, t.cpt, wide_shape(t.cpt, t.groups))) return false;
  const Smem s = smem_layout(pl, K, n_comp, n_slots, t.pp, t.cpt, t.groups);
  if (s.total > smem_optin) return false;
  *out = s;
  return true;
}

// The tuned shape for (K, P) when one is set and valid, else the widest pass that fits
// with the default pairs per thread.
int smem_plan(const Plan& pl, int K, int n_comp, int n_slots, int smem_optin, Smem* out) {
  const int mode = pl.nacc > 0 ? MODE_NORMAL : MODE_MODEL;
  if (mode == MODE_NORMAL) {
    TuneShape t = {0, 0, 0};
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(std::make_pair(K, pl.dd.P));
      if (it != g_tune.end()) t = it->second;
    }
    if (t.pp > 0 && shape_ok(pl, K, n_comp, n_slots, smem_optin, mode, t, out)) {
      g_last_shape = t;
      return GM_OK;
    }
  }
  const int cpt = pick_cpt(pl);
  for (int pp = std::min(kMaxPassPairs, pl.ncp); pp >= 1; --pp) {
    const TuneShape t = {pp, cpt, (pp + cpt - 1) / cpt};
    if (shape_ok(pl, K, n_comp, n_slots, smem_optin, mode, t, out)) {
      g_last_shape = t;
      return GM_OK;
    }
  }
  const Smem s1 = smem_layout(pl, K, n_comp, n_slots, 1, cpt, 1);
  return fail(GM_E_UNSUPPORTED, "tile needs %d bytes of shared memory (K=%d, %d channels); the device allows %d",
              s1.total, K, pl.nch_conv, smem_optin);
}

struct DevInfo {
  int sms = 0, smem_optin = 0;
};

// Fills the nu_n node table of the current device on the first call there
// (k_nu_table, k_nu_ready, then a stream synchronisation so that no other
// stream can see a partial table).  While the caller's stream is being
// captured into a graph it does nothing: set-up kernels then solve nu_n
// directly, which gives the same constants.
std::mutex g_nu_mu;
std::set<int> g_nu_devices;

int ensure_nu_table(cudaStream_t st) {
  int dev = 0;
  GM_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(g_nu_mu);
    if (g_nu_devices.count(dev)) return GM_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GM_CUDA(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) return GM_OK;
  k_nu_table<<<16, 256, 0, st>>>();
  GM_LAUNCHED("k_nu_table");
  k_nu_ready<<<1, 1, 0, st>>>();
  GM_LAUNCHED("k_nu_ready");
  GM_CUDA(cudaStreamSynchronize(st));
  std::lock_guard<std::mutex> lock(g_nu_mu);
  g_nu_devices.insert(dev);
  return GM_OK;
}

int dev_info(DevInfo* di) {
  int dev = 0;
  GM_CUDA(cudaGetDevice(&dev));
  GM_CUDA(cudaDeviceGetAttribute(&di->sms, cudaDevAttrMultiProcessorCount, dev));
  GM_CUDA(cudaDeviceGetAttribute(&di->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  return GM_OK;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

int encode_fn(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    GM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return fail(GM_E_CUDA, "cuTensorMapEncodeTiled is not available");
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  *out = g_encode;
  return GM_OK;
}

// Pair planes of H x W stamps as a rank-3 FP32 tensor: x = 2*Wp floats
// (interleaved pairs), y = H rows, z = n_planes planes; box = 2*window_pitch(K)
// floats x (32+K-1) rows x 1 plane; zero fill outside.
int encode_planes(CUtensorMap* map, float* base, int H, int W, int K, long long n_planes) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  int rc = encode_fn(&enc);
  if (rc) return rc;
  const int Wp = W + (W & 1), rw = window_pitch(K);
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * Wp), (cuuint64_t)H, (cuuint64_t)n_planes};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * Wp) * 4, (cuuint64_t)(2 * Wp) * 4 * H};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * rw), (cuuint32_t)(kTile + K - 1), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(GM_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return GM_OK;
}

// ---------------------------------------------------------------------------
// batch geometry
// ---------------------------------------------------------------------------
// One class of stamps with the same (H, W, K): its planes are one tensor.
struct ClassInfo {
  int H, W, K, n;
  size_t base;  // first float of the class's planes in the plane buffer
};

struct GeomPlan {
  int G = 0, ncp = 0;
  bool ragged = false;
  int H = 0, W = 0, K = 0;   // equal stamps: the sizes; uneven: the largest of each
  long long n_items = 0;     // (galaxy, tile) items of one pass over every galaxy
  size_t plane_floats = 0;   // size of the pair-plane buffer
  std::vector<ClassInfo> cls;
  // host tables of an uneven batch (built when asked for)
  std::vector<GalGeom> geo;
  std::vector<int> order;
  std::vector<int2> items;
};

size_t round_floats(size_t n) { return (n + 63) / 64 * 64; }  // 256-byte multiples

// Sizes, classes and (tables = true, uneven stamps) the geometry table, the
// processing order (decreasing cost: PSF area, then tiles) and the item list.
int plan_geom(const gm_batch* b, int ncp, bool tables, GeomPlan* gp) {
  int rc = check_sizes(b);
  if (rc) return rc;
  gp->G = b->n_gal;
  gp->ncp = ncp;
  gp->ragged = b->geom != nullptr;
  gp->cls.clear();
  gp->geo.clear();
  gp->order.clear();
  gp->items.clear();
  const long long G = b->n_gal;
  if (!gp->ragged) {
    gp->H = b->H;
    gp->W = b->W;
    gp->K = b->K;
    const GalGeom g1 = uniform_geom(0, b->H, b->W, b->K, ncp);
    gp->n_items = G * g1.n_tiles;
    gp->plane_floats = (size_t)G * ncp * b->H * g1.Wp * 2;
    gp->cls.push_back(ClassInfo{b->H, b->W, b->K, (int)G, 0});
  } else {
    std::map<std::tuple<int, int, int>, int> cid;
    std::vector<int> cls_of(tables ? G : 0), rank(tables ? G : 0);
    gp->H = gp->W = gp->K = 1;
    long long items = 0;
    for (long long g = 0; g < G; ++g) {
      const int h = b->geom[3 * g], w = b->geom[3 * g + 1], k = b->geom[3 * g + 2];
      if ((rc = check_hwk(h, w, k, "uneven batch:", (int)g))) return rc;
      auto it = cid.find(std::make_tuple(h, w, k));
      int c;
      if (it == cid.end()) {
        c = (int)gp->cls.size();
        cid.emplace(std::make_tuple(h, w, k), c);
        gp->cls.push_back(ClassInfo{h, w, k, 0, 0});
      } else {
        c = it->second;
      }
      if (tables) {
        cls_of[g] = c;
        rank[g] = gp->cls[c].n;
      }
      ++gp->cls[c].n;
      gp->H = std::max(gp->H, h);
      gp->W = std::max(gp->W, w);
      gp->K = std::max(gp->K, k);
      items += (long long)((w + kTile - 1) / kTile) * ((h + kTile - 1) / kTile);
    }
    gp->n_items = items;
    size_t off = 0;
    for (ClassInfo& c : gp->cls) {
      c.base = off;
      off += round_floats((size_t)c.n * ncp * c.H * (c.W + (c.W & 1)) * 2);
    }
    gp->plane_floats = off;
    if (tables) {
      gp->geo.resize(G);
      long long pix = 0, psf = 0, tile0 = 0;
      for (long long g = 0; g < G; ++g) {
        const ClassInfo& c = gp->cls[cls_of[g]];
        GalGeom r = uniform_geom(0, c.H, c.W, c.K, ncp);
        r.pix = pix;
        r.psf = psf;
        r.plane = (long long)c.base + (long long)rank[g] * ncp * c.H * r.Wp * 2;
        r.tile0 = (int)tile0;
        r.cls = cls_of[g];
        r.z0 = rank[g] * ncp;
        gp->geo[g] = r;
        pix += (long long)c.H * c.W;
        psf += (long long)c.K * c.K;
        tile0 += r.n_tiles;
      }
      gp->order.resize(G);
      for (long long g = 0; g < G; ++g) gp->order[g] = (int)g;
      const std::vector<GalGeom>& geo = gp->geo;
      std::stable_sort(gp->order.begin(), gp->order.end(), [&](int x, int y) {
        if (geo[x].K != geo[y].K) return geo[x].K > geo[y].K;
        return geo[x].n_tiles > geo[y].n_tiles;
      });
      gp->items.reserve(items);
      for (int g : gp->order)
        for (int t = 0; t < geo[g].n_tiles; ++t) gp->items.push_back(make_int2(g, t));
    }
  }
  if (gp->n_items > 0x7fffffffLL)
    return fail(GM_E_UNSUPPORTED, "%lld tiles in one batch exceed 2^31 - 1", gp->n_items);
  return GM_OK;
}

// Workspace shared by the model, chi^2 and fit calls.  geo .. maps are
// adjacent so that an uneven batch's host tables go over in one copy.
struct WsCore {
  size_t geo, order, items, maps, table_end, cconst, scale, psf_pad, planes, partial, err, queue, total;
  int psf_stride;  // floats per galaxy in psf_pad: K psf_row_floats(K) for the batch's largest K
};

WsCore ws_core(const gm_model_desc* d, const GeomPlan& gp, int nacc) {
  WsCore w;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t G = (size_t)std::max(gp.G, 0);
  w.geo = take(G * sizeof(GalGeom));
  w.order = take(G * 4);
  w.items = take((size_t)gp.n_items * 8);
  w.maps = take(gp.ragged ? gp.cls.size() * sizeof(CUtensorMap) : 0);
  w.table_end = off;
  w.cconst = take(G * d->n_comp * kCC * 4);
  w.scale = take(G * scale_stride(d->n_slots) * 4);
  w.psf_stride = gp.K * psf_row_floats(gp.K);  // the largest PSF of the batch (a multiple of 4 floats)
  w.psf_pad = take(G * (size_t)w.psf_stride * 4);
  w.planes = take(gp.plane_floats * 4);
  w.partial = take(nacc > 0 ? (size_t)gp.n_items * nacc * 8 : 0);
  w.err = take(4);
  w.queue = take(4);
  w.total = off;
  return w;
}

struct WsFit {
  WsCore c;
  size_t p_b, p_t, A_b, g_b, chi2_b, lam, pred, it, status, nused, bad, list0, list1, counts, items0, items1,
      icounts, evals, total;
};

WsFit ws_fit(const gm_model_desc* d, const GeomPlan& gp, int P) {
  WsFit w;
  w.c = ws_core(d, gp, 1 + P + P * (P + 1) / 2);
  size_t off = w.c.total;
  const size_t G = (size_t)std::max(gp.G, 0), S = d->n_slots;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  w.p_b = take(G * S * 8);
  w.p_t = take(G * S * 8);
  w.A_b = take(G * (size_t)(P * (P + 1) / 2 + 1) * 8);
  w.g_b = take(G * (size_t)(P + 1) * 8);
  w.chi2_b = take(G * 8);
  w.lam = take(G * 8);
  w.pred = take(G * 8);
  w.it = take(G * 4);
  w.status = take(G * 4);
  w.nused = take(G * 4);
  w.bad = take(G * 4);
  w.list0 = take(G * 4);
  w.list1 = take(G * 4);
  w.counts = take(2 * 4);
  w.items0 = take((size_t)gp.n_items * 8);
  w.items1 = take((size_t)gp.n_items * 8);
  w.icounts = take(2 * 4);
  w.evals = take(3 * 8);
  w.total = off;
  return w;
}

// Kernel arguments that depend only on the model and the shared-memory plan.
void fill_args(FusedArgs& A, const Plan& pl, const Smem& sm) {
  std::memset(&A, 0, sizeof(A));
  A.wait_polls = kWaitTries;
  A.m = chan_map(pl);
  A.nacc = pl.nacc;
  A.pp = sm.pp;
  A.passes = sm.passes;
  A.plane = sm.plane;
  A.off_psf = sm.off_psf;
  A.off_in = sm.off_in;
  A.off_out = sm.off_out;
  A.off_cc = sm.off_cc;
  A.off_scale = sm.off_scale;
  A.off_red = sm.off_red;
  A.off_bar = sm.off_bar;
  A.off_info = sm.off_info;
}

// Geometry table, processing order, the item list of a pass over every galaxy
// and the tensor maps of the planes: built on the device for equal stamps (one
// map, passed by value), copied from the host for uneven ones (one map per
// class, in the workspace).
int put_tables(const GeomPlan& gp, const WsCore& w, char* ws, const DevInfo& di, cudaStream_t st, FusedArgs* A) {
  float* planes = (float*)(ws + w.planes);
  GalGeom* geo = (GalGeom*)(ws + w.geo);
  int* order = (int*)(ws + w.order);
  int2* items = (int2*)(ws + w.items);
  A->geo = geo;
  if (!gp.ragged) {
    const long long n = std::max<long long>(gp.n_items, gp.G);
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * di.sms));
    k_geom_uniform<<<blocks, 256, 0, st>>>(gp.G, gp.H, gp.W, gp.K, gp.ncp, geo, order, items);
    GM_LAUNCHED("k_geom_uniform");
    A->maps = nullptr;
    return encode_planes(&A->tmap, planes, gp.H, gp.W, gp.K, (long long)gp.G * gp.ncp);
  }
  thread_local std::vector<unsigned char> stage;
  stage.assign(w.table_end, 0);
  std::memcpy(stage.data() + w.geo, gp.geo.data(), gp.geo.size() * sizeof(GalGeom));
  std::memcpy(stage.data() + w.order, gp.order.data(), gp.order.size() * sizeof(int));
  std::memcpy(stage.data() + w.items, gp.items.data(), gp.items.size() * sizeof(int2));
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(stage.data() + w.maps);
  for (size_t c = 0; c < gp.cls.size(); ++c) {
    const ClassInfo& ci = gp.cls[c];
    int rc = encode_planes(&maps[c], planes + ci.base, ci.H, ci.W, ci.K, (long long)ci.n * gp.ncp);
    if (rc) return rc;
  }
  GM_CUDA(cudaMemcpyAsync(ws, stage.data(), w.table_end, cudaMemcpyHostToDevice, st));
  A->maps = (const CUtensorMap*)(ws + w.maps);
  return GM_OK;
}

// Profile-kernel arguments of the adjoint path (equal stamps).
ProfileArgs profile_args(const Plan& pl, const gm_batch* b, const float* cconst, const float* scale,
                         float* planes, int Wp) {
  ProfileArgs P;
  std::memset(&P, 0, sizeof(P));
  P.m = chan_map(pl);
  P.G = b->n_gal;
  P.H = b->H;
  P.W = b->W;
  P.Wp = Wp;
  P.cconst = cconst;
  P.scale = scale;
  P.planes = planes;
  return P;
}

PlaneArgs plane_args(const Plan& pl, const GalGeom* geo, const float* cconst, const float* scale, float* planes) {
  PlaneArgs P;
  std::memset(&P, 0, sizeof(P));
  P.m = chan_map(pl);
  P.geo = geo;
  P.cconst = cconst;
  P.scale = scale;
  P.planes = planes;
  return P;
}

int prepare_fused(int mode, const Plan& pl, const Smem& sm, FusedKernel* out) {
  FusedKernel k = pick_kernel(mode, pl.dd.P, sm.cpt, wide_shape(sm.cpt, sm.groups));
  if (!k) return fail(GM_E_UNSUPPORTED, "no fused kernel for %d free parameters", pl.dd.P);
  GM_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm.total));
  *out = k;
  return GM_OK;
}

// Channel pairs the fused pass of `mode` correlates for this description
// (MODEL mode sized for per-component images).
int pairs_for(const gm_model_desc* d, int mode) {
  bool touches_conv[kMaxSlots] = {};
  int n_conv = 0;
  for (int c = 0; c < d->n_comp; ++c) {
    if (!d->comp[c].convolve) continue;
    ++n_conv;
    const int np = comp_np(d, c);
    for (int k = 0; k < np; ++k) touches_conv[d->comp[c].slot[k]] = true;
  }
  int Pc = 0;
  for (int s = 0; s < d->n_slots; ++s) Pc += (d->is_free[s] && touches_conv[s]) ? 1 : 0;
  const int nch = (mode == MODE_NORMAL) ? 1 + Pc : 1 + n_conv;
  return (nch + 1) / 2;
}

int count_free(const gm_model_desc* d) {
  int P = 0;
  for (int s = 0; s < d->n_slots && s < GM_MAX_SLOTS; ++s) P += d->is_free[s] ? 1 : 0;
  return P;
}

int n_acc(int P) { return 1 + P + P * (P + 1) / 2; }

LMOpts lm_opts(const gm_fit_opts* o) {
  LMOpts L;
  std::memset(&L, 0, sizeof(L));  // zero padding: the options are part of the fit graph's key
  if (o) {
    L.tol = o->tol;
    L.xtol = o->xtol;
    L.gtol = o->gtol;
    L.max_iter = o->max_iter;
    L.lambda0 = o->lambda0;
    L.lambda_up = o->lambda_up;
    L.lambda_down = o->lambda_down;
    L.lambda_min = o->lambda_min;
    L.lambda_max = o->lambda_max;
    L.polish = o->polish;
    L.canonical = o->canonical;
    L.lambda_inout = o->lambda_inout;
  } else {
    L.tol = 1e-6;
    L.xtol = 1e-10;
    L.gtol = 1e-10;
    L.max_iter = 100;
    L.lambda0 = 0.1;
    L.lambda_up = 10.0;
    L.lambda_down = 0.2;
    L.lambda_min = 1e-7;
    L.lambda_max = 1e10;
    L.polish = 1;
    L.canonical = 1;
    L.lambda_inout = nullptr;
  }
  return L;
}

// Each galaxy's PSF as the fused kernel holds it in shared memory: K rows of
// psf_row_floats(K) floats, tap t of row a at a * psf_row_floats(K) + 3 cpad + t
// (cpad = ((K-1)/2) & 1), zeros elsewhere.
__global__ void k_psf_pad(int G, const GalGeom* __restrict__ geo, const float* __restrict__ psf, int stride,
                          float* out) {
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    const int K = geo[g].K, KF = psf_row_floats(K), cpad = ((K - 1) / 2) & 1;
    const float* p = psf + geo[g].psf;
    for (int e = threadIdx.x; e < K * KF; e += blockDim.x) {
      const int a = e / KF, t = e - a * KF - 3 * cpad;
      out[(size_t)g * stride + e] = (t >= 0 && t < K) ? p[a * K + t] : 0.f;
    }
  }
}

int launch_psf_pad(int G, const GalGeom* geo, const float* psf, const WsCore& w, char* ws, const DevInfo& di,
                   cudaStream_t st, FusedArgs* A) {
  A->psf_pad = (const float*)(ws + w.psf_pad);
  A->psf_stride = w.psf_stride;
  k_psf_pad<<<std::max(1, std::min(G, 8 * di.sms)), 256, 0, st>>>(G, geo, psf, w.psf_stride,
                                                                    (float*)(ws + w.psf_pad));
  GM_LAUNCHED("k_psf_pad");
  return GM_OK;
}

// LM iterations per CUDA-graph replay in gm_fit_batch (and between convergence polls).
constexpr int kGraphIters = 4;

// Ends a capture left open by an error and frees the graph of one gm_fit_batch call.
struct GraphGuard {
  cudaStream_t capturing = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~GraphGuard() {
    if (capturing) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(capturing, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

// Everything the launches of a fit graph take: a graph captured from these
// values replays the same launches.
struct FitGraphKey {
  PlaneArgs PA;
  FusedArgs A;
  DescDev dd;
  LMState S;
  LMOpts O;
  const void* kf;
  size_t smem;
  int U, G, grid, pgrid, threads, dev;
  cudaEvent_t ev[4 * kGraphIters];
};

// The calling thread's last two fit graphs, each replayed by a later gm_fit_batch whose
// key matches byte for byte (the same model, options, batch buffers and workspace: a
// fit repeated on new data in the same buffers, or alternating between two input
// sets): that call skips the capture and the instantiation of the graph.  `valid` is
// set only once a fit has run the graph to its end without an error.
struct FitGraphCache {
  FitGraphKey key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool valid = false;
  void clear() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    valid = false;
  }
};
thread_local FitGraphCache g_fit_graph[2];
thread_local int g_fit_graph_last = 0;  // the entry used most recently

// A stream of the current device used only to record the fit graph (the
// caller's stream may be the legacy default stream, which cannot capture).
int capture_stream(cudaStream_t* out) {
  constexpr int kDevs = 64;
  thread_local cudaStream_t streams[kDevs] = {};
  int dev = 0;
  GM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kDevs) return fail(GM_E_UNSUPPORTED, "device ordinal %d beyond %d", dev, kDevs);
  if (!streams[dev]) GM_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
  *out = streams[dev];
  return GM_OK;
}

// One model+Jacobian pass over every galaxy (gm_model: MODE_MODEL;
// gm_chi2_grad: MODE_NORMAL, tile partials in the workspace).
struct PassCall {
  Plan pl;
  GeomPlan gp;
  WsCore w;
  Smem sm;
  FusedKernel kf;
  FusedArgs A;
  PlaneArgs PA;
  DevInfo di;
};

int setup_pass(int mode, const gm_model_desc* desc, const gm_batch* batch, const double* params, void* workspace,
               size_t ws_bytes, cudaStream_t st, PassCall* pc) {
  char* ws = (char*)workspace;
  const int G = batch->n_gal;
  pc->w = ws_core(desc, pc->gp, pc->pl.nacc);
  if (!workspace || ws_bytes < pc->w.total)
    return fail(GM_E_NOMEM, "workspace %zu bytes < %zu needed", ws_bytes, pc->w.total);
  int rc;
  if ((rc = dev_info(&pc->di))) return rc;
  if ((rc = smem_plan(pc->pl, pc->gp.K, desc->n_comp, desc->n_slots, pc->di.smem_optin, &pc->sm))) return rc;
  if ((rc = prepare_fused(mode, pc->pl, pc->sm, &pc->kf))) return rc;
  fill_args(pc->A, pc->pl, pc->sm);
  if ((rc = put_tables(pc->gp, pc->w, ws, pc->di, st, &pc->A))) return rc;
  if ((rc = launch_psf_pad(G, pc->A.geo, batch->psf, pc->w, ws, pc->di, st, &pc->A))) return rc;
  FusedArgs& A = pc->A;
  float* cconst = (float*)(ws + pc->w.cconst);
  float* scale = (float*)(ws + pc->w.scale);
  float* planes = (float*)(ws + pc->w.planes);
  A.items = (const int2*)(ws + pc->w.items);
  A.n_items = (int)pc->gp.n_items;
  A.queue = (int*)(ws + pc->w.queue);
  A.image = batch->image;
  A.sigma = batch->sigma;
  A.mask = batch->mask;
  A.psf = batch->psf;
  A.cconst = cconst;
  A.scale = scale;
  A.partial = (double*)(ws + pc->w.partial);
  A.err = (int*)(ws + pc->w.err);
  pc->PA = plane_args(pc->pl, A.geo, cconst, scale, planes);
  pc->PA.items = A.items;
  pc->PA.n_items = A.n_items;
  pc->PA.zero[0] = A.queue;
  GM_CUDA(cudaMemsetAsync(A.err, 0, sizeof(int), st));
  if ((rc = ensure_nu_table(st))) return rc;
  k_setup<<<(G + 31) / 32, 32, 0, st>>>(pc->pl.dd, G, A.geo, 0, 0, params, 0, cconst, scale);
  GM_LAUNCHED("k_setup");
  return GM_OK;
}

int launch_pass(int mode, PassCall* pc, cudaStream_t st) {
  const long long n = pc->gp.n_items;
  const int pgrid = (int)std::max<long long>(1, std::min<long long>(kPlaneUnits * (long long)n, 8LL * pc->di.sms));
  if (mode == MODE_MODEL) k_planes<MODE_MODEL><<<pgrid, 256, 0, st>>>(pc->PA);
  else k_planes<MODE_NORMAL><<<pgrid, 256, 0, st>>>(pc->PA);
  GM_LAUNCHED("k_planes");
  const int grid = (int)std::max<long long>(1, std::min<long long>(n, pc->di.sms));
  FusedArgs A = pc->A;
  if (take_starve(&A.wait_polls)) A.starve = 1;
  pc->kf<<<grid, pc->sm.threads, pc->sm.total, st>>>(A);
  GM_LAUNCHED("k_fused");
  return GM_OK;
}

// Every element of a and b set to NaN when *err is set (a tile load of the pass timed out).
__global__ void k_nan_if_err(const int* __restrict__ err, float* a, size_t na, float* b, size_t nb) {
  if (!*err) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
    if (i < na) a[i] = CUDART_NAN_F;
    else b[i - na] = CUDART_NAN_F;
  }
}

}  // namespace

extern "C" {

int gm_version(void) { return 100; }

int gm_fit_last_stats(gm_fit_stats* out) {
  if (!out) return fail(GM_E_INVAL, "out is NULL");
  if (!g_have_stats) return fail(GM_E_INVAL, "no gm_fit_batch has completed on this thread");
  *out = g_stats;
  return GM_OK;
}

const char* gm_last_error(void) { return g_err; }

int gm_test_starve_next_pass(uint32_t polls) {
  g_starve_polls = polls;
  return GM_OK;
}

int gm_tune_set(int32_t K, int32_t P, int32_t pairs_per_pass, int32_t pairs_per_thread, int32_t groups) {
  if (K < 1 || K > 63 || (K % 2) == 0) return fail(GM_E_INVAL, "gm_tune_set: K=%d must be odd, 1..63", K);
  if (P < 0 || P > GM_MAX_FREE) return fail(GM_E_INVAL, "gm_tune_set: P=%d outside 0..%d", P, GM_MAX_FREE);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (pairs_per_pass == 0) {
    g_tune.erase(std::make_pair(K, P));
    return GM_OK;
  }
  if (!shape_valid(pairs_per_pass, pairs_per_thread, groups))
    return fail(GM_E_INVAL, "gm_tune_set: shape (%d pairs/pass, %d pairs/thread, %d groups) is not a launch shape",
                pairs_per_pass, pairs_per_thread, groups);
  g_tune[std::make_pair(K, P)] = TuneShape{pairs_per_pass, pairs_per_thread, groups};
  return GM_OK;
}

int gm_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  return GM_OK;
}

int gm_tune_last_shape(int32_t* pairs_per_pass, int32_t* pairs_per_thread, int32_t* groups) {
  if (!pairs_per_pass || !pairs_per_thread || !groups) return fail(GM_E_INVAL, "gm_tune_last_shape: NULL output");
  if (g_last_shape.pp == 0) return fail(GM_E_INVAL, "gm_tune_last_shape: no pass planned on this thread yet");
  *pairs_per_pass = g_last_shape.pp;
  *pairs_per_thread = g_last_shape.cpt;
  *groups = g_last_shape.groups;
  return GM_OK;
}

size_t gm_model_workspace_bytes(const gm_model_desc* desc, const gm_batch* batch) {
  if (!desc || !batch || check_desc(desc)) return 0;
  GeomPlan gp;
  if (plan_geom(batch, pairs_for(desc, MODE_MODEL), false, &gp)) return 0;
  return ws_core(desc, gp, 0).total;
}

int gm_model(const gm_model_desc* desc, const gm_batch* batch, const double* params, float* model_out,
             float* comp_out, void* workspace, size_t ws_bytes, void* stream) {
  int rc = check_batch(batch, false);
  if (rc) return rc;
  PassCall pc;
  if ((rc = make_plan(desc, MODE_MODEL, comp_out != nullptr, &pc.pl))) return rc;
  if ((rc = plan_geom(batch, pc.pl.ncp, true, &pc.gp))) return rc;
  if (batch->n_gal == 0) return GM_OK;
  if (!params || !model_out) return fail(GM_E_INVAL, "params/model_out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = setup_pass(MODE_MODEL, desc, batch, params, workspace, ws_bytes, st, &pc))) return rc;
  pc.A.model_out = model_out;
  pc.A.comp_out = comp_out;
  if ((rc = launch_pass(MODE_MODEL, &pc, st))) return rc;
  size_t npix = (size_t)batch->n_gal * (size_t)batch->H * (size_t)batch->W;
  if (batch->geom) {
    npix = 0;
    for (int g = 0; g < batch->n_gal; ++g) npix += (size_t)batch->geom[3 * g] * (size_t)batch->geom[3 * g + 1];
  }
  k_nan_if_err<<<4 * pc.di.sms, 256, 0, st>>>(pc.A.err, model_out, npix, comp_out,
                                               comp_out ? npix * (size_t)desc->n_comp : 0);
  GM_LAUNCHED("k_nan_if_err");
  return GM_OK;
}

size_t gm_chi2_grad_workspace_bytes(const gm_model_desc* desc, const gm_batch* batch) {
  if (!desc || !batch || check_desc(desc)) return 0;
  GeomPlan gp;
  if (plan_geom(batch, pairs_for(desc, MODE_NORMAL), false, &gp)) return 0;
  return ws_core(desc, gp, n_acc(count_free(desc))).total;
}

int gm_chi2_grad(const gm_model_desc* desc, const gm_batch* batch, const double* params, double* chi2,
                 double* grad, double* jtj, void* workspace, size_t ws_bytes, void* stream) {
  int rc = check_batch(batch, true);
  if (rc) return rc;
  PassCall pc;
  if ((rc = make_plan(desc, MODE_NORMAL, false, &pc.pl))) return rc;
  if ((rc = plan_geom(batch, pc.pl.ncp, true, &pc.gp))) return rc;
  if (batch->n_gal == 0) return GM_OK;
  if (!params || !chi2) return fail(GM_E_INVAL, "params/chi2 is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = setup_pass(MODE_NORMAL, desc, batch, params, workspace, ws_bytes, st, &pc))) return rc;
  if ((rc = launch_pass(MODE_NORMAL, &pc, st))) return rc;
  const int G = batch->n_gal;
  k_chi2_grad_finish<<<(G + kLmWarps - 1) / kLmWarps, 32 * kLmWarps, 0, st>>>(pc.pl.dd, G, pc.A.geo, pc.A.partial,
                                                                                pc.A.err, chi2, grad, jtj);
  GM_LAUNCHED("k_chi2_grad_finish");
  return GM_OK;
}

size_t gm_fit_workspace_bytes(const gm_model_desc* desc, const gm_batch* batch) {
  if (!desc || !batch || check_desc(desc)) return 0;
  GeomPlan gp;
  if (plan_geom(batch, pairs_for(desc, MODE_NORMAL), false, &gp)) return 0;
  return ws_fit(desc, gp, count_free(desc)).total;
}

int gm_fit_batch(const gm_model_desc* desc, const gm_batch* batch, double* params_inout, const gm_fit_opts* opts,
                 double* chi2_out, int32_t* dof_out, int32_t* iters_out, int32_t* status_out, double* sigma_p_out,
                 void* workspace, size_t ws_bytes, void* stream) {
  int rc = check_batch(batch, true);
  if (rc) return rc;
  Plan pl;
  if ((rc = make_plan(desc, MODE_NORMAL, false, &pl))) return rc;
  GeomPlan gp;
  if ((rc = plan_geom(batch, pl.ncp, true, &gp))) return rc;
  if (batch->n_gal == 0) return GM_OK;
  if (!params_inout || !chi2_out || !dof_out || !iters_out || !status_out)
    return fail(GM_E_INVAL, "an output pointer is NULL");
  const LMOpts O = lm_opts(opts);
  if (O.max_iter < 1) return fail(GM_E_INVAL, "max_iter=%d < 1", O.max_iter);
  if (O.polish != 0 && O.polish != 1) return fail(GM_E_INVAL, "polish=%d must be 0 or 1", O.polish);
  if (O.canonical != 0 && O.canonical != 1) return fail(GM_E_INVAL, "canonical=%d must be 0 or 1", O.canonical);
  if (!(O.lambda_up > 1.0) || !(O.lambda_down > 0.0) || !(O.lambda_down < 1.0) || !(O.lambda0 > 0.0))
    return fail(GM_E_INVAL, "lambda controls must satisfy lambda0 > 0, up > 1, 0 < down < 1");
  const WsFit w = ws_fit(desc, gp, pl.dd.P);
  if (!workspace || ws_bytes < w.total) return fail(GM_E_NOMEM, "workspace %zu bytes < %zu needed", ws_bytes, w.total);
  DevInfo di;
  if ((rc = dev_info(&di))) return rc;
  Smem sm;
  if ((rc = smem_plan(pl, gp.K, desc->n_comp, desc->n_slots, di.smem_optin, &sm))) return rc;
  FusedKernel kf;
  if ((rc = prepare_fused(MODE_NORMAL, pl, sm, &kf))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  float* cconst = (float*)(ws + w.c.cconst);
  float* scale = (float*)(ws + w.c.scale);
  float* planes = (float*)(ws + w.c.planes);
  int* err = (int*)(ws + w.c.err);
  int* queue = (int*)(ws + w.c.queue);
  double* partial = (double*)(ws + w.c.partial);
  LMState S;
  S.p_b = (double*)(ws + w.p_b);
  S.p_t = (double*)(ws + w.p_t);
  S.A_b = (double*)(ws + w.A_b);
  S.g_b = (double*)(ws + w.g_b);
  S.chi2_b = (double*)(ws + w.chi2_b);
  S.lam = (double*)(ws + w.lam);
  S.pred = (double*)(ws + w.pred);
  S.it = (int*)(ws + w.it);
  S.status = (int*)(ws + w.status);
  S.nused = (int*)(ws + w.nused);
  S.bad = (int*)(ws + w.bad);
  S.list[0] = (int*)(ws + w.list0);
  S.list[1] = (int*)(ws + w.list1);
  S.count[0] = (int*)(ws + w.counts);
  S.count[1] = S.count[0] + 1;
  S.items[0] = (int2*)(ws + w.items0);
  S.items[1] = (int2*)(ws + w.items1);
  S.icount[0] = (int*)(ws + w.icounts);
  S.icount[1] = S.icount[0] + 1;
  S.evals = (unsigned long long*)(ws + w.evals);
  const int G = batch->n_gal;
  const auto t_start = std::chrono::steady_clock::now();
  g_have_stats = false;
  while ((int)g_events.size() < 4 * kGraphIters) {
    cudaEvent_t e;
    GM_CUDA(cudaEventCreate(&e));
    g_events.push_back(e);
  }

  FusedArgs A;
  fill_args(A, pl, sm);
  if ((rc = put_tables(gp, w.c, ws, di, st, &A))) return rc;
  if ((rc = launch_psf_pad(G, A.geo, batch->psf, w.c, ws, di, st, &A))) return rc;
  A.queue = queue;
  A.image = batch->image;
  A.sigma = batch->sigma;
  A.mask = batch->mask;
  A.psf = batch->psf;
  A.cconst = cconst;
  A.scale = scale;
  A.partial = partial;
  A.err = err;
  const int* order = (const int*)(ws + w.c.order);

  GM_CUDA(cudaMemsetAsync(S.evals, 0, 3 * sizeof(unsigned long long), st));
  GM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  GM_CUDA(cudaMemsetAsync(S.count[0], 0, 2 * sizeof(int), st));
  GM_CUDA(cudaMemsetAsync(S.icount[0], 0, 2 * sizeof(int), st));
  k_validate<<<std::min(G, 4 * di.sms), 256, 0, st>>>(G, A.geo, batch->image, batch->sigma, batch->mask, S.nused,
                                                      S.bad);
  GM_LAUNCHED("k_validate");
  if ((rc = ensure_nu_table(st))) return rc;
  k_lm_init<<<(G + 31) / 32, 32, 0, st>>>(pl.dd, S, O, G, A.geo, order, params_inout, cconst, scale);
  GM_LAUNCHED("k_lm_init");

  PlaneArgs PA = plane_args(pl, A.geo, cconst, scale, planes);
  const int grid = (int)std::max<long long>(1, std::min<long long>(gp.n_items, di.sms));
  const int pgrid = (int)std::max<long long>(1, std::min<long long>(kPlaneUnits * gp.n_items, 8LL * di.sms));
  // U iterations captured once as a CUDA graph and replayed, one convergence poll per
  // replay.  U is even (or covers max_iter in one replay), so every replay starts on list 0.
  const int U = std::min(kGraphIters, O.max_iter);
  unsigned starve_polls = 0;
  const bool starve = take_starve(&starve_polls);  // a timeout test: this graph is not kept
  FitGraphKey key;
  std::memset(&key, 0, sizeof(key));
  std::memcpy(&key.PA, &PA, sizeof(PA));
  std::memcpy(&key.A, &A, sizeof(A));
  std::memcpy(&key.dd, &pl.dd, sizeof(pl.dd));
  std::memcpy(&key.S, &S, sizeof(S));
  std::memcpy(&key.O, &O, sizeof(O));
  key.kf = (const void*)kf;
  key.smem = sm.total;
  key.U = U;
  key.G = G;
  key.grid = grid;
  key.pgrid = pgrid;
  key.threads = sm.threads;
  GM_CUDA(cudaGetDevice(&key.dev));
  for (int e = 0; e < 4 * U; ++e) key.ev[e] = g_events[e];
  int slot = -1;
  for (int i = 0; i < 2 && !starve; ++i)
    if (g_fit_graph[i].valid && std::memcmp(&g_fit_graph[i].key, &key, sizeof(key)) == 0) slot = i;
  const bool hit = slot >= 0;
  if (!hit) slot = g_fit_graph_last ^ 1;  // replace the entry used least recently
  g_fit_graph_last = slot;
  FitGraphCache& fc = g_fit_graph[slot];
  fc.valid = false;  // until this call has run the graph without an error
  GraphGuard gg;
  if (!hit) {
    fc.clear();
    cudaStream_t cap;
    if ((rc = capture_stream(&cap))) return rc;
    GM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    gg.capturing = cap;
    for (int u = 0; u < U; ++u) {
      const int cur = u & 1;
      A.items = PA.items = S.items[cur];
      A.n_items_dev = PA.n_items_dev = S.icount[cur];
      PA.zero[0] = queue;
      PA.zero[1] = S.count[cur ^ 1];
      PA.zero[2] = S.icount[cur ^ 1];
      GM_CUDA(cudaEventRecordWithFlags(g_events[4 * u], cap, cudaEventRecordExternal));
      k_planes<MODE_NORMAL><<<pgrid, 256, 0, cap>>>(PA);
      GM_LAUNCHED("k_planes");
      GM_CUDA(cudaEventRecordWithFlags(g_events[4 * u + 1], cap, cudaEventRecordExternal));
      FusedArgs Au = A;
      if (u == 0 && starve) {
        Au.wait_polls = starve_polls;
        Au.starve = 1;
      }
      kf<<<grid, sm.threads, sm.total, cap>>>(Au);
      GM_LAUNCHED("k_fused(normal)");
      GM_CUDA(cudaEventRecordWithFlags(g_events[4 * u + 2], cap, cudaEventRecordExternal));
      k_lm_step<<<(G + kLmGals - 1) / kLmGals, 32 * kLmGals, 0, cap>>>(pl.dd, S, O, cur, A.geo, partial, cconst,
                                                                         scale);
      GM_LAUNCHED("k_lm_step");
      GM_CUDA(cudaEventRecordWithFlags(g_events[4 * u + 3], cap, cudaEventRecordExternal));
    }
    gg.capturing = nullptr;
    GM_CUDA(cudaStreamEndCapture(cap, &gg.graph));
    GM_CUDA(cudaGraphInstantiate(&gg.exec, gg.graph, 0));
    if (!starve) {  // the cache owns it from here
      std::memcpy(&fc.key, &key, sizeof(key));
      fc.graph = gg.graph;
      fc.exec = gg.exec;
      gg.graph = nullptr;
      gg.exec = nullptr;
    }
  }
  const cudaGraphExec_t exec = starve ? gg.exec : fc.exec;
  int passes = 0;
  double profile_ms = 0.0, fused_ms = 0.0, step_ms = 0.0;
  for (int k = 0; k < O.max_iter; k += U) {
    GM_CUDA(cudaGraphLaunch(exec, st));
    passes += U;
    int remaining = 0, kerr = 0;
    GM_CUDA(cudaMemcpyAsync(&remaining, S.count[U & 1], sizeof(int), cudaMemcpyDeviceToHost, st));
    GM_CUDA(cudaMemcpyAsync(&kerr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GM_CUDA(cudaStreamSynchronize(st));
    for (int u = 0; u < U; ++u) {
      float a = 0.f, b = 0.f, c = 0.f;
      GM_CUDA(cudaEventElapsedTime(&a, g_events[4 * u], g_events[4 * u + 1]));
      GM_CUDA(cudaEventElapsedTime(&b, g_events[4 * u + 1], g_events[4 * u + 2]));
      GM_CUDA(cudaEventElapsedTime(&c, g_events[4 * u + 2], g_events[4 * u + 3]));
      profile_ms += a;
      fused_ms += b;
      step_ms += c;
    }
    if (kerr) return fail(GM_E_TIMEOUT, "fused kernel: a tile load did not complete within its wait limit");
    if (remaining == 0) break;
  }
  fc.valid = !starve;
  k_lm_finish<<<(G + kLmGals - 1) / kLmGals, 32 * kLmGals, 0, st>>>(pl.dd, S, G, O.canonical, O.lambda_inout,
                                                                     params_inout, chi2_out, dof_out, iters_out,
                                                                     status_out, sigma_p_out);
  GM_LAUNCHED("k_lm_finish");
  unsigned long long counters[3] = {0, 0, 0};
  GM_CUDA(cudaMemcpyAsync(counters, S.evals, sizeof(counters), cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  gm_fit_stats fs;
  fs.passes = passes;
  fs.graph_reused = hit ? 1 : 0;
  fs.galaxy_evals = (int64_t)counters[0];
  fs.converged = (int64_t)counters[1];
  fs.iters_sum = (int64_t)counters[2];
  fs.profile_ms = profile_ms;
  fs.fused_ms = fused_ms;
  fs.step_ms = step_ms;
  fs.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  g_stats = fs;
  g_have_stats = true;
  return GM_OK;
}

// ---------------------------------------------------------------------------
// adjoint gradient
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

typedef void (*AdjKernel)(AdjArgs);


typedef void (*PixKernel)(PixArgs);

PixKernel pick_resid(int P) {
#define GM_X(PP) \
  if (P == PP) return k_adj_resid<PP>;
  GM_RESID_ALL(GM_X)
#undef GM_X
  return nullptr;
}

PixKernel pick_deriv(int P) {
#define GM_X(PP) \
  if (P == PP) return k_adj_deriv<PP>;
  GM_DERIV_ALL(GM_X)
#undef GM_X
  return nullptr;
}

struct WsAdj {
  size_t cconst, scale, mplanes, uplanes, part_r, part_a, err, total;
  int Wp;
};

WsAdj ws_adj(const gm_model_desc* d, const gm_batch* b, int P) {
  WsAdj w;
  size_t off = 0;
  const size_t G = (size_t)std::max(b->n_gal, 0);
  const size_t pairs = (G + 1) / 2;
  w.Wp = b->W + (b->W & 1);
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  w.cconst = take(G * d->n_comp * kCC * 4);
  w.scale = take(G * scale_stride(d->n_slots) * 4);
  w.mplanes = take(pairs * b->H * w.Wp * 8);
  w.uplanes = take(pairs * b->H * w.Wp * 8);
  // the pixel kernels' sums, per galaxy and part of its stamp
  const size_t parts = (size_t)pix_parts(std::max(b->H, 0), std::max(b->W, 0));
  w.part_r = take(G * parts * (1 + P) * 8);
  w.part_a = take(G * parts * (1 + P) * 8);
  w.err = take(4);
  w.total = off;
  return w;
}

// One planned adjoint pass (gm_grad_adjoint, gm_fit_adam): arguments of both tile
// kernels with their tensor maps, the profile kernel and the launch shape.
struct AdjPass {
  Plan pl;
  WsAdj w;
  AdjArgs Ar, Aa;  // correlations: RESID over the I_conv planes, GRAD over the u = w r planes
  AdjKernel kr, ka;
  PixArgs Xr, Xd;  // pixel kernels: residuals over the M_conv planes, derivative sums over the v planes
  PixKernel kres, kd;  // kd: nullptr without free parameters
  ProfileArgs PA;
  int grid, pgrid, smem;
  char* ws;
};

int prepare_adjoint(const gm_model_desc* desc, const gm_batch* batch, void* workspace, size_t ws_bytes, AdjPass* ap) {
  int rc = check_batch(batch, true);
  if (rc) return rc;
  if (batch->geom) return fail(GM_E_UNSUPPORTED, "the adjoint gradient takes equal stamps only (batch.geom must be NULL)");
  Plan& pl = ap->pl;
  if ((rc = make_plan(desc, MODE_NORMAL, false, &pl))) return rc;
  if (batch->n_gal == 0) return GM_OK;
  const int P = pl.dd.P;
  ap->w = ws_adj(desc, batch, P);
  const WsAdj& w = ap->w;
  if (!workspace || ws_bytes < w.total) return fail(GM_E_NOMEM, "workspace %zu bytes < %zu needed", ws_bytes, w.total);
  DevInfo di;
  if ((rc = dev_info(&di))) return rc;
  const int G = batch->n_gal, K = batch->K, H = batch->H;
  const int n_pairs = (G + 1) / 2;
  char* ws = (char*)workspace;
  ap->ws = ws;
  float* cconst = (float*)(ws + w.cconst);
  float* scale = (float*)(ws + w.scale);
  float* mplanes = (float*)(ws + w.mplanes);
  float* uplanes = (float*)(ws + w.uplanes);
  // the correlations: RESID reads I_conv (model planes) and writes M_conv to the u planes;
  // k_adj_resid turns M_conv into u = w r in place; GRAD reads u and writes v to the model planes
  AdjArgs& A = ap->Ar;
  std::memset(&A, 0, sizeof(A));
  A.G = G;
  A.H = H;
  A.W = batch->W;
  A.Wp = w.Wp;
  A.K = K;
  A.cpad = ((K - 1) / 2) & 1;
  A.tiles_x = (batch->W + kTile - 1) / kTile;
  A.n_tiles = A.tiles_x * ((H + kTile - 1) / kTile);
  A.rw = window_pitch(K);
  const size_t plane_bytes = ((size_t)(kTile + K - 1) * A.rw * 8 + 127) / 128 * 128;
  A.plane = (int)(plane_bytes / 8);
  A.psf = batch->psf;
  A.err = (int*)(ws + w.err);
  A.wait_polls = kWaitTries;
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    const size_t o = off;
    off += bytes;
    return (int)o;
  };
  A.off_in = take(plane_bytes, 128);
  A.off_psf = take((size_t)K * (K + 1) * 8 + 16, 16);  // + the last chunk's prefetch slack
  A.off_bar = take(16, 16);
  ap->smem = (int)off;
  if (ap->smem > di.smem_optin) return fail(GM_E_UNSUPPORTED, "adjoint tile needs %d bytes of shared memory", ap->smem);
  ap->kr = k_adjoint<ADJ_RESID>;
  ap->ka = k_adjoint<ADJ_GRAD>;
  ap->kres = pick_resid(P);
  ap->kd = P > 0 ? pick_deriv(P) : nullptr;
  if (!ap->kres || (P > 0 && !ap->kd)) return fail(GM_E_UNSUPPORTED, "no adjoint kernel for %d free parameters", P);
  GM_CUDA(cudaFuncSetAttribute((const void*)ap->kr, cudaFuncAttributeMaxDynamicSharedMemorySize, ap->smem));
  GM_CUDA(cudaFuncSetAttribute((const void*)ap->ka, cudaFuncAttributeMaxDynamicSharedMemorySize, ap->smem));
  int occ = 1;
  GM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)ap->kr, 128, ap->smem));
  ap->grid = std::max(1, std::min(n_pairs * A.n_tiles, std::max(occ, 1) * di.sms));
  ap->PA = profile_args(pl, batch, cconst, scale, mplanes, w.Wp);
  ap->pgrid = std::max(1, std::min(n_pairs * ((H * w.Wp + 255) / 256), 8 * di.sms));
  A.out_planes = uplanes;
  if ((rc = encode_planes(&A.tmap, mplanes, H, batch->W, K, n_pairs))) return rc;
  ap->Aa = A;
  ap->Aa.out_planes = mplanes;
  if ((rc = encode_planes(&ap->Aa.tmap, uplanes, H, batch->W, K, n_pairs))) return rc;
  // the pixel kernels
  PixArgs X;
  std::memset(&X, 0, sizeof(X));
  X.m = chan_map(pl);
  X.G = G;
  X.H = H;
  X.W = batch->W;
  X.Wp = w.Wp;
  X.tiles_x = A.tiles_x;
  X.n_tiles = A.n_tiles;
  X.image = batch->image;
  X.sigma = batch->sigma;
  X.mask = batch->mask;
  X.cconst = cconst;
  ap->Xr = X;
  ap->Xd = X;
  for (int c = 0; c < desc->n_comp; ++c)
    for (int k = 0; k < 8; ++k) {
      const int f = (k < pl.dd.np[c]) ? pl.chan_of_slot[pl.dd.slot[c][k]] - 1 : -1;
      ap->Xr.acc_of[c][k] = pl.conv[c] ? -1 : f;
      ap->Xd.acc_of[c][k] = pl.conv[c] ? f : -1;
    }
  ap->Xr.planes = uplanes;
  ap->Xr.partial = (double*)(ws + w.part_r);
  ap->Xd.planes = mplanes;
  ap->Xd.partial = (double*)(ws + w.part_a);
  return GM_OK;
}

// chi^2 and d chi^2/dp at params: set-up, profile planes, both correlations, per-galaxy sums.
int launch_adjoint(const AdjPass& ap, const gm_batch* batch, const double* params, double* chi2, double* grad,
                   cudaStream_t st, const cudaEvent_t* ev = nullptr) {
  const int G = batch->n_gal;
  auto mark = [&](int k) -> int {
    if (ev) GM_CUDA(cudaEventRecord(ev[k], st));
    return GM_OK;
  };
  int rc;
  if ((rc = mark(0))) return rc;
  if (int rc = ensure_nu_table(st)) return rc;
  k_setup<<<(G + 31) / 32, 32, 0, st>>>(ap.pl.dd, G, nullptr, batch->H, batch->W, params, 0,
                                        (float*)(ap.ws + ap.w.cconst), (float*)(ap.ws + ap.w.scale));
  GM_LAUNCHED("k_setup");
  k_profile_pairs<<<ap.pgrid, 256, 0, st>>>(ap.PA);
  GM_LAUNCHED("k_profile_pairs");
  if ((rc = mark(1))) return rc;
  const int n_parts = pix_parts(batch->H, batch->W), blocks = (G + 1) / 2 * n_parts;
  AdjArgs Ar = ap.Ar;
  if (take_starve(&Ar.wait_polls)) Ar.starve = 1;
  ap.kr<<<ap.grid, 128, ap.smem, st>>>(Ar);
  GM_LAUNCHED("k_adjoint(resid)");
  if ((rc = mark(2))) return rc;
  ap.kres<<<blocks, kPixThreads, 0, st>>>(ap.Xr);
  GM_LAUNCHED("k_adj_resid");
  if ((rc = mark(3))) return rc;
  ap.ka<<<ap.grid, 128, ap.smem, st>>>(ap.Aa);
  GM_LAUNCHED("k_adjoint(grad)");
  if ((rc = mark(4))) return rc;
  if (ap.kd) {
    ap.kd<<<blocks, kPixThreads, 0, st>>>(ap.Xd);
    GM_LAUNCHED("k_adj_deriv");
  } else {
    GM_CUDA(cudaMemsetAsync(ap.Xd.partial, 0, (size_t)G * n_parts * (1 + ap.pl.dd.P) * 8, st));
  }
  // the pixel kernels leave one partial per galaxy and part of its stamp
  k_adjoint_finish<<<(G + 127) / 128, 128, 0, st>>>(ap.pl.dd, G, n_parts, ap.Xr.partial, ap.Xd.partial, ap.Ar.err,
                                                    chi2, grad);
  GM_LAUNCHED("k_adjoint_finish");
  return mark(5);
}

// Workspace of gm_fit_adam: the adjoint pass's, then the current point, its chi^2
// and gradient, and the Adam moments and step scales.
struct WsAdamState {
  WsAdj adj;
  size_t cur, grad, chi2, m, v, scale, total;
};

WsAdamState ws_adam(const gm_model_desc* d, const gm_batch* b, int P) {
  WsAdamState w;
  w.adj = ws_adj(d, b, P);
  size_t off = w.adj.total;
  const size_t G = (size_t)std::max(b->n_gal, 0), S = d->n_slots;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  w.cur = take(G * S * 8);
  w.grad = take(G * S * 8);
  w.chi2 = take(G * 8);
  w.m = take(G * S * 8);
  w.v = take(G * S * 8);
  w.scale = take(G * S * 8);
  w.total = off;
  return w;
}

}  // namespace

extern "C" {

size_t gm_grad_adjoint_workspace_bytes(const gm_model_desc* desc, const gm_batch* batch) {
  if (!desc || !batch || check_desc(desc) || check_sizes(batch) || batch->geom) return 0;
  return ws_adj(desc, batch, count_free(desc)).total;
}

int gm_grad_adjoint(const gm_model_desc* desc, const gm_batch* batch, const double* params, double* chi2,
                    double* grad, void* workspace, size_t ws_bytes, void* stream) {
  AdjPass ap;
  int rc = prepare_adjoint(desc, batch, workspace, ws_bytes, &ap);
  if (rc || batch->n_gal == 0) return rc;
  if (!params || !chi2) return fail(GM_E_INVAL, "params/chi2 is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  GM_CUDA(cudaMemsetAsync(ap.Ar.err, 0, sizeof(int), st));
  // kernel timing events, unless the stream is being captured into a graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  GM_CUDA(cudaStreamIsCapturing(st, &cs));
  g_adj_timed = false;
  const cudaEvent_t* ev = nullptr;
  if (cs == cudaStreamCaptureStatusNone) {
    for (auto& e : g_adj_events)
      if (!e) GM_CUDA(cudaEventCreate(&e));
    ev = g_adj_events;
  }
  if ((rc = launch_adjoint(ap, batch, params, chi2, grad, st, ev))) return rc;
  g_adj_timed = ev != nullptr;
  return GM_OK;
}

int gm_grad_adjoint_last_stats(gm_adjoint_stats* out) {
  if (!out) return fail(GM_E_INVAL, "out is NULL");
  if (!g_adj_timed) return fail(GM_E_INVAL, "no timed gm_grad_adjoint call on this thread");
  GM_CUDA(cudaEventSynchronize(g_adj_events[5]));
  float t[5];
  for (int k = 0; k < 5; ++k) GM_CUDA(cudaEventElapsedTime(&t[k], g_adj_events[k], g_adj_events[k + 1]));
  out->setup_ms = t[0];
  out->resid_ms = t[1];
  out->residual_ms = t[2];
  out->grad_ms = t[3];
  out->deriv_ms = t[4];
  return GM_OK;
}

size_t gm_fit_adam_workspace_bytes(const gm_model_desc* desc, const gm_batch* batch) {
  if (!desc || !batch || check_desc(desc) || check_sizes(batch) || batch->geom) return 0;
  return ws_adam(desc, batch, count_free(desc)).total;
}

int gm_fit_adam(const gm_model_desc* desc, const gm_batch* batch, double* params_inout, const gm_adam_opts* opts,
                double* chi2_out, void* workspace, size_t ws_bytes, void* stream) {
  if (!opts) return fail(GM_E_INVAL, "opts is NULL");
  if (opts->n_iter < 1 || !(opts->lr > 0.0) || !(opts->beta1 >= 0.0 && opts->beta1 < 1.0) ||
      !(opts->beta2 >= 0.0 && opts->beta2 < 1.0) || !(opts->eps > 0.0))
    return fail(GM_E_INVAL, "Adam options need n_iter >= 1, lr > 0, 0 <= beta < 1, eps > 0");
  if (!desc || !batch) return fail(GM_E_INVAL, "desc/batch is NULL");
  const WsAdamState wa = ws_adam(desc, batch, count_free(desc));
  if (!workspace || ws_bytes < wa.total) return fail(GM_E_NOMEM, "workspace %zu bytes < %zu needed", ws_bytes, wa.total);
  AdjPass ap;
  int rc = prepare_adjoint(desc, batch, workspace, wa.adj.total, &ap);
  if (rc || batch->n_gal == 0) return rc;
  if (!params_inout || !chi2_out) return fail(GM_E_INVAL, "params/chi2 is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const int G = batch->n_gal, NS = desc->n_slots;
  double* cur = (double*)(ws + wa.cur);
  double* grad = (double*)(ws + wa.grad);
  double* chi2 = (double*)(ws + wa.chi2);
  AdamState S;
  S.m = (double*)(ws + wa.m);
  S.v = (double*)(ws + wa.v);
  S.scale = (double*)(ws + wa.scale);
  S.best = params_inout;
  S.best_chi2 = chi2_out;
  GM_CUDA(cudaMemsetAsync(ap.Ar.err, 0, sizeof(int), st));
  if (int rc = ensure_nu_table(st)) return rc;
  k_adam_init<<<(G + 127) / 128, 128, 0, st>>>(ap.pl.dd, G, params_inout, cur, S);
  GM_LAUNCHED("k_adam_init");
  for (int t = 1; t <= opts->n_iter; ++t) {
    if ((rc = launch_adjoint(ap, batch, cur, chi2, grad, st))) return rc;
    const double c1 = 1.0 - std::pow(opts->beta1, (double)t), c2 = 1.0 - std::pow(opts->beta2, (double)t);
    k_adam_step<<<(G + 127) / 128, 128, 0, st>>>(ap.pl.dd, G, cur, grad, chi2, S, opts->lr, opts->beta1, opts->beta2,
                                                 opts->eps, c1, c2, t == opts->n_iter ? 1 : 0);
    GM_LAUNCHED("k_adam_step");
  }
  // the last step's point, then the best point seen, canonical
  if ((rc = launch_adjoint(ap, batch, cur, chi2, grad, st))) return rc;
  k_adam_finish<<<(G + 127) / 128, 128, 0, st>>>(ap.pl.dd, G, cur, chi2, S);
  GM_LAUNCHED("k_adam_finish");
  int kerr = 0;
  GM_CUDA(cudaMemcpyAsync(&kerr, ap.Ar.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  if (kerr) return fail(GM_E_TIMEOUT, "adjoint kernel: a tile load did not complete within its wait limit");
  (void)NS;
  return GM_OK;
}

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// bootstrap (Sec. 5.2): pixels resampled with replacement, refits, scatter
// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): the finaliser of a Weyl sequence with
// increment 0x9E3779B97F4A7C15; used as a counter-based generator.
__host__ __device__ inline unsigned long long splitmix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Draw k of replicate b for galaxy g: the (k+1)-th output of the SplitMix64
// stream whose state starts at splitmix64(splitmix64(seed) ^ (g << 32 | b)).
__device__ inline unsigned long long boot_draw(unsigned long long seed, unsigned long long g, unsigned long long b,
                                               unsigned long long k) {
  const unsigned long long key = splitmix64(splitmix64(seed) ^ ((g << 32) | b));
  return splitmix64(key + (k + 1) * 0x9E3779B97F4A7C15ull);
}

// Row-major list of each galaxy's unmasked pixels and their number (one block per galaxy).
__global__ void k_boot_compact(int G, int HW, const uint8_t* __restrict__ mask, int* list, int* n_used) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int t0 = 0; t0 < HW; t0 += blockDim.x) {
      const int t = t0 + threadIdx.x;
      const bool used = t < HW && !(mask && mask[(size_t)g * HW + t]);
      const unsigned bal = __ballot_sync(0xffffffffu, used);
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      if (lane == 0) s_warp[warp] = __popc(bal);
      __syncthreads();
      int before = s_base;
      for (int w = 0; w < warp; ++w) before += s_warp[w];
      if (used) list[(size_t)g * HW + before + __popc(bal & ((1u << lane) - 1u))] = t;
      __syncthreads();
      if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s_base += s_warp[w];
      __syncthreads();
    }
    if (threadIdx.x == 0) n_used[g] = s_base;
    __syncthreads();
  }
}

// Multiplicity of each pixel in replicate b: n_used draws, uniform over the unmasked pixels.
__global__ void k_boot_draw(int G, int HW, const int* __restrict__ list, const int* __restrict__ n_used,
                            unsigned long long seed, int b, unsigned* counts) {
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    const unsigned long long N = (unsigned long long)n_used[g];
    for (unsigned long long k = threadIdx.x; k < N; k += blockDim.x) {
      const unsigned long long r = boot_draw(seed, (unsigned long long)g, (unsigned long long)b, k);
      const int idx = (int)__umul64hi(r, N);  // floor(r N / 2^64)
      atomicAdd(&counts[(size_t)g * HW + list[(size_t)g * HW + idx]], 1u);
    }
  }
}

// The replicate as a batch: sigma / sqrt(count) on drawn pixels, masked where the count is 0.
__global__ void k_boot_weights(long long n, const float* __restrict__ sigma, const uint8_t* __restrict__ mask,
                               const unsigned* __restrict__ counts, float* sigma_eff, uint8_t* mask_eff) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const unsigned c = counts[t];
    const bool off = c == 0u || (mask && mask[t]);
    mask_eff[t] = off ? 1 : 0;
    sigma_eff[t] = off ? 1.f : sigma[t] * rsqrtf((float)c);
  }
}

// Running mean and sum of squared deviations (Welford) of the converged refits;
// position angles taken within pi/2 of the best fit's.
__global__ void k_boot_accum(const __grid_constant__ DescDev D, int G, const double* __restrict__ pb,
                             const int* __restrict__ status, const double* __restrict__ best, double* mean,
                             double* m2, int* n_ok) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G || status[g] != ST_CONVERGED) return;
  const int NS = D.n_slots;
  const int n = ++n_ok[g];
  const double pi = 3.14159265358979323846;
  for (int s = 0; s < NS; ++s) {
    double x = pb[(size_t)g * NS + s];
    if (D.is_pa[s]) {
      const double ref = best[(size_t)g * NS + s];
      x = ref + (x - ref) - pi * floor((x - ref) / pi + 0.5);
    }
    const size_t e = (size_t)g * NS + s;
    const double d = x - mean[e];
    mean[e] += d / n;
    m2[e] += d * (x - mean[e]);
  }
}

__global__ void k_boot_finish(int n, const double* __restrict__ m2, const int* __restrict__ n_ok, int NS,
                              double* sigma_boot) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int c = n_ok[e / NS];
  sigma_boot[e] = c > 0 ? sqrt(m2[e] / c) : CUDART_NAN;  // (1/M) sum (p_i - mean)^2 (Sec. 5.2)
}

struct WsBoot {
  size_t fit, list, n_used, counts, sigma_eff, mask_eff, pb, chi2, dof, iters, status, mean, m2, n_ok, total;
  size_t fit_bytes;
};

WsBoot ws_boot(const gm_model_desc* d, const gm_batch* b) {
  WsBoot w;
  w.fit_bytes = gm_fit_workspace_bytes(d, b);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t G = (size_t)std::max(b->n_gal, 0), N = G * (size_t)b->H * b->W, S = d->n_slots;
  w.fit = take(w.fit_bytes);
  w.list = take(N * 4);
  w.n_used = take(G * 4);
  w.counts = take(N * 4);
  w.sigma_eff = take(N * 4);
  w.mask_eff = take(N);
  w.pb = take(G * S * 8);
  w.chi2 = take(G * 8);
  w.dof = take(G * 4);
  w.iters = take(G * 4);
  w.status = take(G * 4);
  w.mean = take(G * S * 8);
  w.m2 = take(G * S * 8);
  w.n_ok = take(G * 4);
  w.total = off;
  return w;
}

// Counts of replicate b into ws counts (list and n_used already built).
int boot_counts(const gm_batch* batch, const WsBoot& w, char* ws, unsigned long long seed, int b, cudaStream_t st) {
  const int G = batch->n_gal, HW = batch->H * batch->W;
  GM_CUDA(cudaMemsetAsync(ws + w.counts, 0, (size_t)G * HW * 4, st));
  k_boot_draw<<<std::max(1, std::min(G, 1184)), 256, 0, st>>>(G, HW, (const int*)(ws + w.list),
                                                              (const int*)(ws + w.n_used), seed, b,
                                                              (unsigned*)(ws + w.counts));
  GM_LAUNCHED("k_boot_draw");
  return GM_OK;
}

int boot_check(const gm_model_desc* desc, const gm_batch* batch) {
  int rc = check_batch(batch, true);
  if (rc) return rc;
  if ((rc = check_desc(desc))) return rc;
  if (batch->geom) return fail(GM_E_UNSUPPORTED, "the bootstrap takes equal stamps only (batch.geom must be NULL)");
  return GM_OK;
}

}  // namespace

extern "C" {

size_t gm_bootstrap_workspace_bytes(const gm_model_desc* desc, const gm_batch* batch) {
  if (!desc || !batch || check_desc(desc) || check_sizes(batch) || batch->geom) return 0;
  return ws_boot(desc, batch).total;
}

int gm_bootstrap_counts(const gm_model_desc* desc, const gm_batch* batch, uint64_t seed, int32_t replicate,
                        uint32_t* counts, void* workspace, size_t ws_bytes, void* stream) {
  int rc = boot_check(desc, batch);
  if (rc) return rc;
  if (batch->n_gal == 0) return GM_OK;
  if (!counts || replicate < 0) return fail(GM_E_INVAL, "counts is NULL or replicate < 0");
  const WsBoot w = ws_boot(desc, batch);
  if (!workspace || ws_bytes < w.total) return fail(GM_E_NOMEM, "workspace %zu bytes < %zu needed", ws_bytes, w.total);
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const int G = batch->n_gal, HW = batch->H * batch->W;
  k_boot_compact<<<std::max(1, std::min(G, 1184)), 256, 0, st>>>(G, HW, batch->mask, (int*)(ws + w.list),
                                                                 (int*)(ws + w.n_used));
  GM_LAUNCHED("k_boot_compact");
  if ((rc = boot_counts(batch, w, ws, seed, replicate, st))) return rc;
  GM_CUDA(cudaMemcpyAsync(counts, ws + w.counts, (size_t)G * HW * 4, cudaMemcpyDeviceToDevice, st));
  return GM_OK;
}

int gm_bootstrap(const gm_model_desc* desc, const gm_batch* batch, const double* params_best, int32_t n_boot,
                 uint64_t seed, const gm_fit_opts* opts, double* sigma_boot, int32_t* n_ok, void* workspace,
                 size_t ws_bytes, void* stream) {
  int rc = boot_check(desc, batch);
  if (rc) return rc;
  if (batch->n_gal == 0) return GM_OK;
  if (!params_best || !sigma_boot || n_boot < 1) return fail(GM_E_INVAL, "params_best/sigma_boot NULL or n_boot < 1");
  const WsBoot w = ws_boot(desc, batch);
  if (!workspace || ws_bytes < w.total) return fail(GM_E_NOMEM, "workspace %zu bytes < %zu needed", ws_bytes, w.total);
  Plan pl;
  if ((rc = make_plan(desc, MODE_NORMAL, false, &pl))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const int G = batch->n_gal, HW = batch->H * batch->W, NS = desc->n_slots;
  const long long N = (long long)G * HW;
  double* pb = (double*)(ws + w.pb);
  double* mean = (double*)(ws + w.mean);
  double* m2 = (double*)(ws + w.m2);
  int* nok = (int*)(ws + w.n_ok);
  GM_CUDA(cudaMemsetAsync(mean, 0, (size_t)G * NS * 8, st));
  GM_CUDA(cudaMemsetAsync(m2, 0, (size_t)G * NS * 8, st));
  GM_CUDA(cudaMemsetAsync(nok, 0, (size_t)G * 4, st));
  k_boot_compact<<<std::max(1, std::min(G, 1184)), 256, 0, st>>>(G, HW, batch->mask, (int*)(ws + w.list),
                                                                 (int*)(ws + w.n_used));
  GM_LAUNCHED("k_boot_compact");
  gm_batch rep = *batch;
  rep.sigma = (const float*)(ws + w.sigma_eff);
  rep.mask = (const uint8_t*)(ws + w.mask_eff);
  // every replicate's refit starts fresh and returns canonical parameters (PA aligned below)
  gm_fit_opts ropts;
  const gm_fit_opts* ropts_p = nullptr;
  if (opts) {
    ropts = *opts;
    ropts.canonical = 1;
    ropts.lambda_inout = nullptr;
    ropts_p = &ropts;
  }
  const int ngrid = (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, 4096));
  for (int b = 0; b < n_boot; ++b) {
    if ((rc = boot_counts(batch, w, ws, (unsigned long long)seed, b, st))) return rc;
    k_boot_weights<<<ngrid, 256, 0, st>>>(N, batch->sigma, batch->mask, (const unsigned*)(ws + w.counts),
                                          (float*)(ws + w.sigma_eff), (uint8_t*)(ws + w.mask_eff));
    GM_LAUNCHED("k_boot_weights");
    GM_CUDA(cudaMemcpyAsync(pb, params_best, (size_t)G * NS * 8, cudaMemcpyDeviceToDevice, st));
    if ((rc = gm_fit_batch(desc, &rep, pb, ropts_p, (double*)(ws + w.chi2), (int32_t*)(ws + w.dof),
                           (int32_t*)(ws + w.iters), (int32_t*)(ws + w.status), nullptr, ws + w.fit, w.fit_bytes,
                           stream)))
      return rc;
    k_boot_accum<<<(G + 127) / 128, 128, 0, st>>>(pl.dd, G, pb, (const int*)(ws + w.status), params_best, mean, m2,
                                                  nok);
    GM_LAUNCHED("k_boot_accum");
  }
  k_boot_finish<<<(G * NS + 255) / 256, 256, 0, st>>>(G * NS, m2, nok, NS, sigma_boot);
  GM_LAUNCHED("k_boot_finish");
  if (n_ok) GM_CUDA(cudaMemcpyAsync(n_ok, nok, (size_t)G * 4, cudaMemcpyDeviceToDevice, st));
  return GM_OK;
}

}  // extern "C"

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per
// device with that device current.
int noalloc_scratch(void** out) {
  int dev = 0;
  GM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(GM_E_UNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(GM_E_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) on device %d: %s", dev, cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GM_OK;
}

}  // namespace

extern "C" int gm_chi2_grad_noalloc(const gm_model_desc* desc, const gm_batch* batch, const double* params,
                                    double* chi2, double* grad, double* jtj, void* stream) {
  int rc = check_batch(batch, true);
  if (rc) return rc;
  if ((rc = check_desc(desc))) return rc;
  // the geometry is planned here rather than through the size query, so that a
  // refusal keeps plan_geom's own reason in the error message
  GeomPlan gp;
  if ((rc = plan_geom(batch, pairs_for(desc, MODE_NORMAL), false, &gp))) return rc;
  if (batch->n_gal == 0) return GM_OK;  // no device call, as for every other entry point
  const size_t need = ws_core(desc, gp, n_acc(count_free(desc))).total;
  if (need > (size_t)GM_NOALLOC_SCRATCH_BYTES)
    return fail(GM_E_NOMEM,
                "gm_chi2_grad_noalloc: this batch needs %zu bytes of scratch but the built-in array holds %u; "
                "split the batch or call gm_chi2_grad with your own workspace",
                need, (unsigned)GM_NOALLOC_SCRATCH_BYTES);
  void* ws = nullptr;
  if ((rc = noalloc_scratch(&ws))) return rc;
  return gm_chi2_grad(desc, batch, params, chi2, grad, jtj, ws, (size_t)GM_NOALLOC_SCRATCH_BYTES, stream);
}
