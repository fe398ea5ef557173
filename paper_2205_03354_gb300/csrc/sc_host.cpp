// Exact stencil algebra on the host: the 1D stencils the paper prints,
// embedding into d dimensions, sums, composition (Sec. 2.2, Eq. C=B(A)) and
// correctly rounded floating-point weights.  Everything here is integer
// arithmetic on (offset, numerator) lists over a common denominator; nothing
// touches the device.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <vector>

#include "sc_internal.h"

namespace sc {

static thread_local char g_err[512] = "";

int fail(int status, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return status;
}

void clear_error() { g_err[0] = 0; }

static int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

static int bitlen(u128 v) {
  int n = 0;
  while (v) {
    v >>= 1;
    ++n;
  }
  return n;
}

double round_ratio(bool neg, u128 n, u128 d, int P) {
  if (n == 0) return neg ? -0.0 : 0.0;
  // e = floor(log2(n/d))
  int e = bitlen(n) - bitlen(d);
  bool ge;
  if (e >= 0)
    ge = n >= (d << e);
  else
    ge = (n << (-e)) >= d;
  if (!ge) --e;
  // scale so that nn/dd lies in [1, 2)
  u128 nn = n, dd = d;
  if (e >= 0)
    dd = d << e;
  else
    nn = n << (-e);
  // long division: P significand bits, then one guard bit and a sticky bit
  uint64_t q = 0;
  for (int i = 0; i < P; ++i) {
    uint64_t bit = nn >= dd;
    if (bit) nn -= dd;
    q = (q << 1) | bit;
    nn <<= 1;
  }
  bool guard = nn >= dd;
  if (guard) nn -= dd;
  bool sticky = nn != 0;
  if (guard && (sticky || (q & 1))) {
    ++q;
    if (q == (uint64_t(1) << P)) {
      q >>= 1;
      ++e;
    }
  }
  double v = std::ldexp(double(q), e - (P - 1));
  return neg ? -v : v;
}

// num/den * (h_den/h_num)^p as an exact ratio n/d with sign.
static int exact_weight(int64_t num, int64_t den, int hp, int64_t h_num, int64_t h_den,
                        bool *neg, u128 *n, u128 *d) {
  *neg = num < 0;
  u128 a = (u128)(num < 0 ? -(i128)num : (i128)num);
  u128 b = (u128)den;
  u128 sn = 1, sd = 1;
  int p = hp < 0 ? -hp : hp;
  const u128 lim = ((u128)1) << 126;
  for (int i = 0; i < p; ++i) {
    if (sn > lim / (u128)h_den || sd > lim / (u128)h_num)
      return fail(SC_EOVERFLOW, "h^-%d does not fit 126 bits", hp);
    sn *= (u128)h_den;
    sd *= (u128)h_num;
  }
  if (hp < 0) std::swap(sn, sd);
  if (a != 0 && sn > lim / a) return fail(SC_EOVERFLOW, "weight numerator overflow");
  if (sd > lim / b) return fail(SC_EOVERFLOW, "weight denominator overflow");
  *n = a * sn;
  *d = b * sd;
  return SC_OK;
}

int weights_f64(const sc_stencil *s, int64_t h_num, int64_t h_den, double *out) {
  for (int i = 0; i < s->npts; ++i) {
    bool neg;
    u128 n, d;
    int st = exact_weight(s->num[i], s->den, s->hpow, h_num, h_den, &neg, &n, &d);
    if (st) return st;
    out[i] = round_ratio(neg, n, d, 53);
  }
  return SC_OK;
}

int weights_f32(const sc_stencil *s, int64_t h_num, int64_t h_den, float *out) {
  for (int i = 0; i < s->npts; ++i) {
    bool neg;
    u128 n, d;
    int st = exact_weight(s->num[i], s->den, s->hpow, h_num, h_den, &neg, &n, &d);
    if (st) return st;
    double v = round_ratio(neg, n, d, 24);  // exactly representable as float
    if (std::fabs(v) > 3.4028234663852886e38 || (v != 0 && std::fabs(v) < 1.1754943508222875e-38))
      return fail(SC_EOVERFLOW, "weight outside the float normal range");
    out[i] = float(v);
  }
  return SC_OK;
}

// ---- building stencils -----------------------------------------------------

typedef std::array<int32_t, 3> Off;

static bool add_checked(int64_t a, int64_t b, int64_t *r) { return !__builtin_add_overflow(a, b, r); }
static bool mul_checked(int64_t a, int64_t b, int64_t *r) { return !__builtin_mul_overflow(a, b, r); }

// Normalises a map of offsets -> numerators over `den` into `out`.
static int finish(const std::map<Off, int64_t> &m, int64_t den, int ndim, int hpow, sc_stencil *out) {
  int64_t g = den;
  int n = 0;
  for (auto &kv : m)
    if (kv.second != 0) {
      g = gcd64(g, kv.second);
      ++n;
    }
  if (n > SC_MAX_PTS) return fail(SC_EINVAL, "stencil has %d points (max %d)", n, SC_MAX_PTS);
  if (g == 0) g = 1;
  std::memset(out, 0, sizeof(*out));
  out->ndim = ndim;
  out->hpow = hpow;
  out->den = den / g;
  int i = 0, r = 0;
  for (auto &kv : m) {  // std::map iterates offsets in lexicographic order
    if (kv.second == 0) continue;
    for (int a = 0; a < 3; ++a) {
      out->off[i][a] = kv.first[a];
      r = std::max(r, std::abs(kv.first[a]));
    }
    out->num[i] = kv.second / g;
    ++i;
  }
  out->npts = i;
  out->radius = r;
  return SC_OK;
}

static int check(const sc_stencil *s) {
  if (!s) return fail(SC_EINVAL, "null stencil");
  if (s->ndim < 1 || s->ndim > 3) return fail(SC_EINVAL, "ndim %d not in 1..3", s->ndim);
  if (s->npts < 0 || s->npts > SC_MAX_PTS) return fail(SC_EINVAL, "npts %d out of range", s->npts);
  if (s->den <= 0) return fail(SC_EINVAL, "den must be positive");
  return SC_OK;
}

}  // namespace sc

using namespace sc;

extern "C" {

int32_t sc_version(void) { return 100; }

const char *sc_last_error(void) { return sc::g_err; }

int sc_stencil_1d(int32_t kind, sc_stencil *out) {
  if (!out) return fail(SC_EINVAL, "null output");
  std::map<Off, int64_t> m;
  int64_t den = 1;
  int hp = 0;
  auto put = [&](int k, int64_t v) { m[Off{k, 0, 0}] = v; };
  switch (kind) {
    case SC_D1_C2: den = 2; hp = 1; put(1, 1); put(-1, -1); break;
    case SC_D2_C2: den = 1; hp = 2; put(-1, 1); put(0, -2); put(1, 1); break;
    case SC_D1_C4: den = 12; hp = 1; put(1, 8); put(2, -1); put(-2, 1); put(-1, -8); break;
    case SC_D2_C4: den = 12; hp = 2; put(-2, -1); put(-1, 16); put(0, -30); put(1, 16); put(2, -1); break;
    case SC_D1_FWD: den = 1; hp = 1; put(1, 1); put(0, -1); break;
    case SC_D2_FWD: den = 1; hp = 2; put(2, 1); put(1, -2); put(0, 1); break;
    default: return fail(SC_EINVAL, "unknown 1D stencil kind %d", kind);
  }
  clear_error();
  return finish(m, den, 1, hp, out);
}

int sc_stencil_embed(const sc_stencil *s, int32_t ndim, int32_t axis, sc_stencil *out) {
  if (int st = check(s)) return st;
  if (!out) return fail(SC_EINVAL, "null output");
  if (s->ndim != 1) return fail(SC_EINVAL, "embed takes a 1D stencil");
  if (ndim < 1 || ndim > 3 || axis < 0 || axis >= ndim) return fail(SC_EINVAL, "bad ndim/axis");
  std::map<Off, int64_t> m;
  for (int i = 0; i < s->npts; ++i) {
    Off o{0, 0, 0};
    o[axis] = s->off[i][0];
    m[o] = s->num[i];
  }
  clear_error();
  return finish(m, s->den, ndim, s->hpow, out);
}

int sc_stencil_add(const sc_stencil *a, const sc_stencil *b, sc_stencil *out) {
  if (int st = check(a)) return st;
  if (int st = check(b)) return st;
  if (!out) return fail(SC_EINVAL, "null output");
  if (a->ndim != b->ndim || a->hpow != b->hpow)
    return fail(SC_EINVAL, "add needs equal ndim and h-power");
  // common denominator: lcm(den_a, den_b)
  int64_t g = gcd64(a->den, b->den);
  int64_t fa = b->den / g, fb = a->den / g, den;
  if (!mul_checked(a->den, fa, &den)) return fail(SC_EOVERFLOW, "denominator overflow");
  std::map<Off, int64_t> m;
  for (int i = 0; i < a->npts; ++i) {
    int64_t v;
    if (!mul_checked(a->num[i], fa, &v)) return fail(SC_EOVERFLOW, "numerator overflow");
    Off o{a->off[i][0], a->off[i][1], a->off[i][2]};
    m[o] = v;
  }
  for (int i = 0; i < b->npts; ++i) {
    int64_t v, t;
    if (!mul_checked(b->num[i], fb, &v)) return fail(SC_EOVERFLOW, "numerator overflow");
    Off o{b->off[i][0], b->off[i][1], b->off[i][2]};
    if (!add_checked(m[o], v, &t)) return fail(SC_EOVERFLOW, "numerator overflow");
    m[o] = t;
  }
  clear_error();
  return finish(m, den, a->ndim, a->hpow, out);
}

int sc_laplacian(int32_t ndim, int32_t order, sc_stencil *out) {
  if (!out) return fail(SC_EINVAL, "null output");
  if (ndim < 1 || ndim > 3) return fail(SC_EINVAL, "ndim %d not in 1..3", ndim);
  if (order != 2 && order != 4) return fail(SC_EINVAL, "order must be 2 or 4");
  sc_stencil base, ax, acc, tmp;
  int st = sc_stencil_1d(order == 2 ? SC_D2_C2 : SC_D2_C4, &base);
  if (st) return st;
  if ((st = sc_stencil_embed(&base, ndim, 0, &acc))) return st;
  for (int a = 1; a < ndim; ++a) {
    if ((st = sc_stencil_embed(&base, ndim, a, &ax))) return st;
    if ((st = sc_stencil_add(&acc, &ax, &tmp))) return st;
    acc = tmp;
  }
  *out = acc;
  clear_error();
  return SC_OK;
}

int sc_compose_stencil(const sc_stencil *outer, const sc_stencil *inner, sc_stencil *out) {
  if (int st = check(outer)) return st;
  if (int st = check(inner)) return st;
  if (!out) return fail(SC_EINVAL, "null output");
  if (out == outer || out == inner) return fail(SC_EINVAL, "output aliases an input");
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "composition needs equal dimensions");
  int64_t den;
  if (!mul_checked(outer->den, inner->den, &den)) return fail(SC_EOVERFLOW, "denominator overflow");
  std::map<Off, int64_t> m;
  for (int j = 0; j < outer->npts; ++j)
    for (int i = 0; i < inner->npts; ++i) {
      Off o;
      for (int a = 0; a < 3; ++a) o[a] = outer->off[j][a] + inner->off[i][a];
      int64_t prod, t;
      if (!mul_checked(outer->num[j], inner->num[i], &prod)) return fail(SC_EOVERFLOW, "product overflow");
      if (!add_checked(m[o], prod, &t)) return fail(SC_EOVERFLOW, "sum overflow");
      m[o] = t;
    }
  clear_error();
  return finish(m, den, outer->ndim, outer->hpow + inner->hpow, out);
}

int sc_stencil_weights(const sc_stencil *s, int64_t h_num, int64_t h_den, int32_t dtype, void *host_out) {
  if (int st = check(s)) return st;
  if (!host_out) return fail(SC_EINVAL, "null output");
  if (h_num <= 0 || h_den <= 0) return fail(SC_EINVAL, "h must be positive");
  int st;
  if (dtype == SC_F64)
    st = weights_f64(s, h_num, h_den, (double *)host_out);
  else if (dtype == SC_F32)
    st = weights_f32(s, h_num, h_den, (float *)host_out);
  else
    return fail(SC_EINVAL, "unknown dtype %d", dtype);
  if (!st) clear_error();
  return st;
}

}  // extern "C"
