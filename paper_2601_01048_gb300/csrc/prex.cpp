// Partial representative execution (Sec. 5.1) of the cufz engine: which
// test threads of an input decide whether any thread of its grid violates.
// Two host analyses over the decoded program, both exact: the corner check
// (the theorem of Sec. 5.1.1, for kernels without thread-dependent
// conditions) and the guarded-grid plan (for kernels whose conditions are
// guards on one launch dimension each, the class of Sec. 5.1's Alg. 1).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ir.h"

namespace cufz {
namespace {

// The corner check.  Theorem (Sec. 5.1.1): in a
// kernel whose access indices are affine in the thread and block indices
// with coefficients shared by all threads, and whose accesses sit under no
// thread-dependent condition, a violating thread exists iff one of the
// corner threads (every thread and block coordinate first or last) violates.
// The check executes the program once on the host over abstract values:
// uniform (one int32 for every thread), affine (exact integer coefficients
// of tid.x/y/z, ctaid.x/y/z plus a constant) or other.  An input qualifies
// when every branch decision and loop trip is uniform, every access index
// is uniform or affine, and no affine value leaves the int32 range anywhere
// in the launch box (the device computes in wrapping 32-bit arithmetic, so
// an index that could wrap would not be affine).

struct AVal {
  uint8_t k = 0;  // 0 uniform, 1 affine, 2 other
  int32_t u = 0;
  int64_t c[6] = {0, 0, 0, 0, 0, 0};
  int64_t b = 0;
};

constexpr int64_t kAffMax = (int64_t)1 << 40;  // coefficient bound of the exact arithmetic

uint32_t host_fmix32(uint32_t h) {  // MurmurHash3 finalizer, as the device's mix32
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

int32_t uniform_alu(int op, int32_t x, int32_t y) {
  const uint32_t ux = (uint32_t)x, uy = (uint32_t)y;
  switch (op) {
    case 0: return (int32_t)(ux + uy);
    case 1: return (int32_t)(ux - uy);
    case 2: return (int32_t)(ux * uy);
    case 3: return (int32_t)(ux << (uy & 31u));
    case 4: return x >> (int)(uy & 31u);
    case 5: return (int32_t)(ux >> (uy & 31u));
    case 6: return (int32_t)(ux & uy);
    case 7: return (int32_t)(ux | uy);
    case 8: return (int32_t)(ux ^ uy);
    case 9: return x < y ? x : y;
    case 10: return x > y ? x : y;
    case 11: return x < y;
    case 12: return x <= y;
    case 13: return x == y;
    case 14: return x != y;
    default: return ux < uy;
  }
}

struct PrexRun {
  const Ir& ir;
  const cufz_input& in;
  uint32_t budget;
  int64_t ext[6];  // largest value of each coordinate
  std::vector<AVal> r;
  uint64_t back = 0;
  bool stopped = false;

  static AVal uni(int32_t x) {
    AVal v;
    v.u = x;
    return v;
  }
  static AVal other() {
    AVal v;
    v.k = 2;
    return v;
  }
  static AVal as_affine(const AVal& x) {
    if (x.k == 1) return x;
    AVal v;
    v.k = 1;
    v.b = x.u;
    return v;
  }
  // Range check of an affine value over the launch box; a value constant
  // over the box becomes uniform.  False when it could leave int32.
  bool norm(AVal& v) const {
    if (v.k != 1) return true;
    if (v.b > kAffMax || v.b < -kAffMax) return false;
    int64_t lo = v.b, hi = v.b;
    for (int k = 0; k < 6; k++) {
      if (v.c[k] > kAffMax || v.c[k] < -kAffMax) return false;
      const int64_t t = v.c[k] * ext[k];
      (t > 0 ? hi : lo) += t;
    }
    if (lo < INT32_MIN || hi > INT32_MAX) return false;
    if (lo == hi) {
      v = uni((int32_t)lo);
    }
    return true;
  }
  static bool scale(AVal& v, int64_t s) {
    for (int k = 0; k < 6; k++) {
      const __int128 p = (__int128)v.c[k] * s;
      if (p > kAffMax || p < -kAffMax) return false;
      v.c[k] = (int64_t)p;
    }
    const __int128 p = (__int128)v.b * s;
    if (p > kAffMax || p < -kAffMax) return false;
    v.b = (int64_t)p;
    return true;
  }
  AVal alu(int op, const AVal& x, const AVal& y) const {
    if (x.k == 0 && y.k == 0) return uni(uniform_alu(op, x.u, y.u));
    if (x.k == 2 || y.k == 2) return other();
    AVal v;
    switch (op) {
      case 0:
      case 1: {
        const AVal a = as_affine(x), b = as_affine(y);
        v.k = 1;
        for (int k = 0; k < 6; k++) v.c[k] = op == 0 ? a.c[k] + b.c[k] : a.c[k] - b.c[k];
        v.b = op == 0 ? a.b + b.b : a.b - b.b;
        return v;
      }
      case 2:
        if (x.k == 1 && y.k == 1) return other();
        v = x.k == 1 ? x : y;
        return scale(v, x.k == 1 ? y.u : x.u) ? v : other();
      case 3:
        if (y.k != 0) return other();
        v = x;
        return scale(v, (int64_t)1 << ((uint32_t)y.u & 31u)) ? v : other();
      default:
        return other();
    }
  }
  AVal sreg(int id) const {
    if (id <= 2 || (id >= 6 && id <= 8)) {
      AVal v;
      v.k = 1;
      v.c[id <= 2 ? id : id - 3] = 1;
      return v;
    }
    if (id <= 5) return uni((int32_t)in.block[id - 3]);
    if (id <= 11) return uni((int32_t)in.grid[id - 9]);
    return uni(in.args[id - 12]);
  }
  // The value a uniform index loads (0 when it violates or the buffer is shared).
  AVal load(const IrOp& o, int32_t idx) const {
    const int64_t w = o.width, off = (int64_t)idx * w;
    const int64_t len = (int64_t)in.buf_len[o.buf];
    if (off < 0 || off + w > len || ((ir.shared_mask >> o.buf) & 1u)) return uni(0);
    const uint32_t word =
        host_fmix32(ir.seed ^ ((uint32_t)o.buf * 0x9E3779B9u) ^ (uint32_t)((uint64_t)off >> 2));
    return uni(w == 1 ? (int32_t)((word >> (8u * ((uint32_t)off & 3u))) & 0xFFu) : (int32_t)word);
  }
  // Executes ops [pc, end); false as soon as the input does not qualify.
  bool exec(int pc, int end) {
    while (pc < end && !stopped) {
      const IrOp& o = ir.ops[pc];
      const uint8_t opc = o.opc;
      if (is_alu_reg(opc) || is_alu_imm(opc)) {
        const bool im = is_alu_imm(opc);
        AVal v = alu(opc - (im ? 0x30 : 0x10), r[o.a], im ? uni(o.imm) : r[o.b]);
        if (!norm(v)) return false;
        r[o.dst] = v;
        pc++;
        continue;
      }
      switch (opc) {
        case B_SREG: {
          AVal v = sreg(o.sreg);
          if (!norm(v)) return false;
          r[o.dst] = v;
          pc++;
          break;
        }
        case B_IMM: r[o.dst] = uni(o.imm); pc++; break;
        case B_MOV: r[o.dst] = r[o.a]; pc++; break;
        case B_SEL: {
          const AVal& cnd = r[o.a];
          if (cnd.k == 0) r[o.dst] = cnd.u ? r[o.b] : r[o.c];
          else if (r[o.b].k == 0 && r[o.c].k == 0 && r[o.b].u == r[o.c].u) r[o.dst] = r[o.b];
          else r[o.dst] = other();
          pc++;
          break;
        }
        case B_LD:
        case B_ST: {
          const AVal idx = r[o.a];
          if (idx.k == 2) return false;  // an index that is neither uniform nor affine
          if (opc == B_LD) r[o.dst] = idx.k == 0 ? load(o, idx.u) : other();
          pc++;
          break;
        }
        case B_IF: {
          if (r[o.a].k != 0) return false;  // a thread-dependent condition
          const int then_end = o.else_pc >= 0 ? o.else_pc : o.end_pc;
          if (r[o.a].u) {
            if (!exec(pc + 1, then_end)) return false;
          } else if (o.else_pc >= 0) {
            if (!exec(o.else_pc + 1, o.end_pc)) return false;
          }
          pc = o.end_pc + 1;
          break;
        }
        case B_LOOP: {
          if (r[o.a].k != 0) return false;  // a thread-dependent trip count
          const int32_t n = r[o.a].u;
          const int32_t trip = n < 0 ? 0 : (n > o.imm ? o.imm : n);
          int32_t k = 0;
          for (; k < trip && !stopped; k++) {
            r[o.dst] = uni(k);
            if (!exec(pc + 1, o.end_pc)) return false;
            if (stopped) break;
            if (++back > budget) stopped = true;  // every thread stops here
          }
          if (!stopped) r[o.dst] = uni(trip);
          pc = o.end_pc + 1;
          break;
        }
        case B_DIV:
        case B_REM:
        case B_HALLOC:
        case B_HFREE:
        case B_HLD:
        case B_HST: return false;  // a division or a heap op: not in either analysis
        default: pc++; break;
      }
    }
    return true;
  }
};


// Guarded kernels (the case Sec. 5.1.2 leaves to the heuristic Alg. 1),
// exactly.  Each launch dimension d is one axis, the global coordinate
// G_d = b_d * n_d + t_d in [0, n_d * g_d), when every access index and
// every compared value depends on (t_d, b_d) only through G_d; otherwise it
// is two axes, t_d in [0, n_d) and b_d in [0, g_d).  A guard compares
// values affine in one dimension's coordinates, so its truth changes only
// at a few *cuts* of that dimension's axes: a cut at v separates v - 1 from
// v.  The cuts of all guards split the launch box into cells (boxes) in
// which every guard, and so every branch condition and loop trip, is
// constant.  In a cell each access index is one affine function of the
// coordinates (or a constant), and an affine function is out of bounds
// somewhere in a box iff it is at one of the box's corners.  So the threads
// whose every axis coordinate is an axis end or next to a cut (v - 1 or v)
// decide the verdict: the plan.
//
// Values are tracked per cell.  A value built from guards and
// thread-invariant values only (a guard, a combination of guards, a load at
// such an index) is constant in each cell.  A value that is one of a few
// affine functions in each cell, the same one throughout the cell, is
// piecewise affine: min and max of affine values (their comparison is a
// guard), a register that the two sides of a guard leave different, a
// selection by a guard.  Both sides of a guard are executed.  A guard on a
// combination of two dimensions (x + y < n) is refused, as is any affine
// piece that could wrap int32, a loop trip that varies between threads, and
// a path that reaches the iteration budget.

struct Aff {
  int64_t ct[3] = {0, 0, 0}, cb[3] = {0, 0, 0}, b = 0;  // sum ct * t_d + cb * b_d + b
  bool constant() const {
    for (int d = 0; d < 3; d++)
      if (ct[d] || cb[d]) return false;
    return true;
  }
  bool operator==(const Aff& o) const {
    for (int d = 0; d < 3; d++)
      if (ct[d] != o.ct[d] || cb[d] != o.cb[d]) return false;
    return b == o.b;
  }
  bool operator<(const Aff& o) const {
    for (int d = 0; d < 3; d++) {
      if (ct[d] != o.ct[d]) return ct[d] < o.ct[d];
      if (cb[d] != o.cb[d]) return cb[d] < o.cb[d];
    }
    return b < o.b;
  }
};

constexpr size_t kMaxForms = 8;  // pieces of a piecewise-affine value

struct GVal {
  // 0 uniform, 1 affine, 2 constant in each cell, 3 other, 4 piecewise
  // affine (one of the forms f in each cell)
  uint8_t k = 0;
  int32_t u = 0;
  std::vector<Aff> f;  // k == 1: one form; k == 4: two or more, sorted
  bool operator==(const GVal& o) const { return k == o.k && u == o.u && f == o.f; }
};

struct PrexGrid {
  const Ir& ir;
  const cufz_input& in;
  uint32_t budget;
  bool merged[3];          // dimension d is one axis G_d
  bool need_split[3] = {false, false, false};
  int64_t n[3], g[3];      // block and grid extents
  std::vector<int64_t> cut_t[3], cut_b[3], cut_g[3];

  static GVal uni(int32_t x) {
    GVal v;
    v.u = x;
    return v;
  }
  static GVal kind(uint8_t k) {
    GVal v;
    v.k = k;
    return v;
  }
  static bool affine_kind(const GVal& v) { return v.k == 0 || v.k == 1 || v.k == 4; }
  static std::vector<Aff> forms(const GVal& v) {
    if (v.k != 0) return v.f;
    Aff a;
    a.b = v.u;
    return {a};
  }
  static int64_t floor_div(int64_t p, int64_t q) {
    int64_t f = p / q;
    if ((p % q != 0) && ((p < 0) != (q < 0))) f--;
    return f;
  }
  static int64_t ceil_div(int64_t p, int64_t q) { return -floor_div(-p, q); }

  // Drops coefficients of coordinates fixed at 0 and checks the int32 range
  // of the form over the launch box.
  bool norm_form(Aff& a) const {
    int64_t lo = a.b, hi = a.b;
    for (int d = 0; d < 3; d++) {
      if (n[d] == 1) a.ct[d] = 0;
      if (g[d] == 1) a.cb[d] = 0;
      for (int64_t c : {a.ct[d], a.cb[d]})
        if (c > kAffMax || c < -kAffMax) return false;
      const int64_t t1 = a.ct[d] * (n[d] - 1), t2 = a.cb[d] * (g[d] - 1);
      (t1 > 0 ? hi : lo) += t1;
      (t2 > 0 ? hi : lo) += t2;
    }
    return a.b <= kAffMax && a.b >= -kAffMax && lo >= INT32_MIN && hi <= INT32_MAX;
  }
  // A value from its possible forms: uniform, affine, piecewise affine, or
  // (all forms constant, several of them) constant in each cell.  False if a
  // form could wrap int32; too many forms make it "other".
  bool from_forms(std::vector<Aff> fs, GVal* out) const {
    for (Aff& a : fs)
      if (!norm_form(a)) return false;
    std::sort(fs.begin(), fs.end());
    fs.erase(std::unique(fs.begin(), fs.end()), fs.end());
    if (fs.empty() || fs.size() > kMaxForms) {
      *out = kind(3);
      return true;
    }
    bool all_const = true;
    for (const Aff& a : fs) all_const = all_const && a.constant();
    if (fs.size() == 1 && all_const) {
      *out = uni((int32_t)fs[0].b);
    } else if (all_const) {
      *out = kind(2);
    } else {
      out->k = fs.size() == 1 ? 1 : 4;
      out->u = 0;
      out->f = std::move(fs);
    }
    return true;
  }
  bool norm(GVal& v) const { return (v.k != 1 && v.k != 4) || from_forms(v.f, &v); }
  // Whether form a depends on dimension d's coordinates only through G_d
  // (and then its coefficient of G_d).
  bool global_form(const Aff& a, int d, int64_t* c) const {
    if (g[d] == 1) {
      *c = a.ct[d];
      return true;
    }
    if (n[d] == 1) {
      *c = a.cb[d];
      return true;
    }
    *c = a.ct[d];
    return a.cb[d] == a.ct[d] * n[d];
  }
  // An access index in a merged dimension must be in global form; otherwise
  // the dimension is split and the analysis runs again.
  bool merge_ok(const GVal& v) {
    bool ok = true;
    for (const Aff& a : v.f)
      for (int d = 0; d < 3; d++) {
        int64_t c = 0;
        if (merged[d] && !global_form(a, d, &c)) {
          need_split[d] = true;
          ok = false;
        }
      }
    return ok;
  }
  // Cuts where "c * x + b op 0" changes along x in [0, m) (c != 0).
  static void add_cuts(std::vector<int64_t>& cuts, int64_t m, int op, int64_t c, int64_t b) {
    auto add = [&](int64_t v) {
      if (v >= 1 && v < m) cuts.push_back(v);
    };
    switch (op) {
      case 11: add(c > 0 ? ceil_div(-b, c) : floor_div(-b, c) + 1); break;  // c x + b < 0
      case 12: add(c > 0 ? floor_div(-b, c) + 1 : ceil_div(-b, c)); break;  // c x + b <= 0
      default:                                                              // == 0, != 0
        if ((-b) % c == 0) {
          add(-b / c);
          add(-b / c + 1);
        }
        break;
    }
  }
  // The guard "a op 0": records its cuts; false when its truth does not
  // follow the axes (two dimensions, or one split dimension through both
  // coordinates other than as G_d).  A constant a needs no cut.
  bool guard(const Aff& a, int op) {
    int dim = -1;
    for (int d = 0; d < 3; d++)
      if (a.ct[d] || a.cb[d]) {
        if (dim >= 0) return false;
        dim = d;
      }
    if (dim < 0) return true;
    const int d = dim;
    int64_t c = 0;
    if (merged[d]) {
      if (!global_form(a, d, &c)) {
        need_split[d] = true;
        return false;
      }
      add_cuts(cut_g[d], n[d] * g[d], op, c, a.b);
      return true;
    }
    if (!a.cb[d]) {
      add_cuts(cut_t[d], n[d], op, a.ct[d], a.b);
      return true;
    }
    if (!a.ct[d]) {
      add_cuts(cut_b[d], g[d], op, a.cb[d], a.b);
      return true;
    }
    if (!global_form(a, d, &c)) return false;
    // a staircase in (t_d, b_d): a cut at G = q * n + r splits block q
    // between threads r - 1 and r, and blocks q - 1 | q | q + 1 apart
    std::vector<int64_t> gc;
    add_cuts(gc, n[d] * g[d], op, c, a.b);
    for (int64_t x : gc) {
      const int64_t q = x / n[d], r = x % n[d];
      if (q >= 1) cut_b[d].push_back(q);
      if (r != 0) {
        cut_t[d].push_back(r);
        if (q + 1 < g[d]) cut_b[d].push_back(q + 1);
      }
    }
    return true;
  }
  // The difference x - y of two forms with the coefficients of fixed
  // coordinates dropped.
  Aff diff(const Aff& x, const Aff& y) const {
    Aff a;
    for (int d = 0; d < 3; d++) {
      a.ct[d] = n[d] == 1 ? 0 : x.ct[d] - y.ct[d];
      a.cb[d] = g[d] == 1 ? 0 : x.cb[d] - y.cb[d];
    }
    a.b = x.b - y.b;
    return a;
  }
  // Guards "p op q" for every pair of forms; false if one is not a guard.
  bool guard_pairs(const std::vector<Aff>& xs, const std::vector<Aff>& ys, int op) {
    for (const Aff& p : xs)
      for (const Aff& q : ys)
        if (!guard(diff(p, q), op)) return false;
    return true;
  }
  static bool scale(Aff& a, int64_t s) {
    for (int64_t* c : {&a.ct[0], &a.ct[1], &a.ct[2], &a.cb[0], &a.cb[1], &a.cb[2], &a.b}) {
      const __int128 p = (__int128)*c * s;
      if (p > kAffMax || p < -kAffMax) return false;
      *c = (int64_t)p;
    }
    return true;
  }
  // The value that is x in some cells and y in the others (a join after a
  // guard, a selection by a guard).
  GVal combine(const GVal& x, const GVal& y) const {
    if (x == y) return x;
    if ((x.k == 0 || x.k == 2) && (y.k == 0 || y.k == 2)) return kind(2);
    if (!affine_kind(x) || !affine_kind(y)) return kind(3);
    std::vector<Aff> fs = forms(x), fy = forms(y);
    fs.insert(fs.end(), fy.begin(), fy.end());
    GVal v;
    return from_forms(fs, &v) ? v : kind(3);
  }
  // Makes a truth value per cell of v (tested against zero); false if that
  // needs a guard that is not one.
  bool truth(GVal& v) {
    if (v.k == 1 || v.k == 4) {
      for (const Aff& a : v.f)
        if (!guard(a, 14)) return false;
      v = kind(2);
    }
    return true;
  }
  GVal alu(int op, const GVal& x, const GVal& y) {
    if (x.k == 0 && y.k == 0) return uni(uniform_alu(op, x.u, y.u));
    if (x.k == 3 || y.k == 3) return kind(3);
    if ((x.k == 0 || x.k == 2) && (y.k == 0 || y.k == 2)) return kind(2);  // cell constants
    if (x.k == 2 || y.k == 2) return kind(3);  // affine with a cell constant
    const std::vector<Aff> fx = forms(x), fy = forms(y);
    std::vector<Aff> out;
    switch (op) {
      case 0:
      case 1:
        for (const Aff& p : fx)
          for (const Aff& q : fy) {
            Aff a = p;
            const int64_t s = op == 0 ? 1 : -1;
            for (int d = 0; d < 3; d++) {
              a.ct[d] += s * q.ct[d];
              a.cb[d] += s * q.cb[d];
            }
            a.b += s * q.b;
            out.push_back(a);
          }
        break;
      case 2:
      case 3: {
        if (y.k != 0 && (op == 3 || x.k != 0)) return kind(3);
        const bool x_scaled = y.k == 0;
        const int64_t s = op == 3 ? (int64_t)1 << ((uint32_t)y.u & 31u) : x_scaled ? y.u : x.u;
        for (Aff a : x_scaled ? fx : fy) {
          if (!scale(a, s)) return kind(3);
          out.push_back(a);
        }
        break;
      }
      case 9:
      case 10:  // min / max: x where x < y holds (a guard per pair), else y
        if (!guard_pairs(fx, fy, 11)) return kind(3);
        out = fx;
        out.insert(out.end(), fy.begin(), fy.end());
        break;
      case 11:
      case 12:
      case 13:
      case 14: {  // a signed comparison of affine values: a guard per pair
        if (fx.size() == 1 && fy.size() == 1) {
          const Aff dv = diff(fx[0], fy[0]);
          if (dv.constant())
            return uni(op == 11 ? dv.b < 0 : op == 12 ? dv.b <= 0 : op == 13 ? dv.b == 0 : dv.b != 0);
        }
        return guard_pairs(fx, fy, op) ? kind(2) : kind(3);
      }
      default:
        return kind(3);
    }
    GVal v;
    return from_forms(out, &v) ? v : kind(3);
  }
  GVal sreg(int id) const {
    GVal v;
    Aff a;
    if (id <= 2) {
      a.ct[id] = 1;
    } else if (id >= 6 && id <= 8) {
      a.cb[id - 6] = 1;
    } else if (id <= 5) {
      return uni((int32_t)in.block[id - 3]);
    } else if (id <= 11) {
      return uni((int32_t)in.grid[id - 9]);
    } else {
      return uni(in.args[id - 12]);
    }
    v.k = 1;
    v.f = {a};
    return v;
  }
  GVal load(const IrOp& o, int32_t idx) const {
    const int64_t w = o.width, off = (int64_t)idx * w;
    const int64_t len = (int64_t)in.buf_len[o.buf];
    if (off < 0 || off + w > len || ((ir.shared_mask >> o.buf) & 1u)) return uni(0);
    const uint32_t word =
        host_fmix32(ir.seed ^ ((uint32_t)o.buf * 0x9E3779B9u) ^ (uint32_t)((uint64_t)off >> 2));
    return uni(w == 1 ? (int32_t)((word >> (8u * ((uint32_t)off & 3u))) & 0xFFu) : (int32_t)word);
  }
  struct State {
    std::vector<GVal> r;
    uint64_t back = 0;
  };
  // Executes [pc, end) on st; false if the input does not qualify.
  bool exec(int pc, int end, State& st) {
    while (pc < end) {
      const IrOp& o = ir.ops[pc];
      const uint8_t opc = o.opc;
      if (is_alu_reg(opc) || is_alu_imm(opc)) {
        const bool im = is_alu_imm(opc);
        GVal v = alu(opc - (im ? 0x30 : 0x10), st.r[o.a], im ? uni(o.imm) : st.r[o.b]);
        if (!norm(v)) return false;
        st.r[o.dst] = v;
        pc++;
        continue;
      }
      switch (opc) {
        case B_SREG: {
          GVal v = sreg(o.sreg);
          if (!norm(v)) return false;
          st.r[o.dst] = v;
          pc++;
          break;
        }
        case B_IMM: st.r[o.dst] = uni(o.imm); pc++; break;
        case B_MOV: st.r[o.dst] = st.r[o.a]; pc++; break;
        case B_SEL: {
          GVal c = st.r[o.a];
          const GVal &x = st.r[o.b], &y = st.r[o.c];
          if (c.k == 0) {
            st.r[o.dst] = c.u ? x : y;
          } else if (x == y) {
            st.r[o.dst] = x;
          } else {
            if (!truth(c)) return false;
            st.r[o.dst] = c.k == 2 ? combine(x, y) : kind(3);
          }
          pc++;
          break;
        }
        case B_LD:
        case B_ST: {
          const GVal idx = st.r[o.a];
          if (idx.k == 3 || !merge_ok(idx)) return false;
          if (opc == B_LD) st.r[o.dst] = idx.k == 0 ? load(o, idx.u) : kind(idx.k == 2 ? 2 : 3);
          pc++;
          break;
        }
        case B_IF: {
          GVal c = st.r[o.a];
          if (!truth(c)) return false;
          const int then_end = o.else_pc >= 0 ? o.else_pc : o.end_pc;
          if (c.k == 0) {
            if (c.u) {
              if (!exec(pc + 1, then_end, st)) return false;
            } else if (o.else_pc >= 0) {
              if (!exec(o.else_pc + 1, o.end_pc, st)) return false;
            }
          } else if (c.k == 2) {
            State a = st, e = st;
            if (!exec(pc + 1, then_end, a)) return false;
            if (o.else_pc >= 0 && !exec(o.else_pc + 1, o.end_pc, e)) return false;
            for (size_t k = 0; k < st.r.size(); k++) st.r[k] = combine(a.r[k], e.r[k]);
            st.back = std::max(a.back, e.back);
          } else {
            return false;
          }
          pc = o.end_pc + 1;
          break;
        }
        case B_LOOP: {
          if (st.r[o.a].k != 0) return false;
          const int32_t nt = st.r[o.a].u;
          const int32_t trip = nt < 0 ? 0 : (nt > o.imm ? o.imm : nt);
          for (int32_t k = 0; k < trip; k++) {
            st.r[o.dst] = uni(k);
            if (!exec(pc + 1, o.end_pc, st)) return false;
            if (++st.back > budget) return false;  // a budget stop: not covered here
          }
          st.r[o.dst] = uni(trip);
          pc = o.end_pc + 1;
          break;
        }
        case B_DIV:
        case B_REM:
        case B_HALLOC:
        case B_HFREE:
        case B_HLD:
        case B_HST: return false;  // a division or a heap op: not in either analysis
        default: pc++; break;
      }
    }
    return true;
  }
};

// Coordinates on one axis that the plan takes: the ends and both sides of
// every cut.
std::vector<int64_t> axis_points(std::vector<int64_t> cuts, int64_t m) {
  std::vector<int64_t> p = {0, m - 1};
  for (int64_t v : cuts) {
    p.push_back(v - 1);
    p.push_back(v);
  }
  std::sort(p.begin(), p.end());
  p.erase(std::unique(p.begin(), p.end()), p.end());
  return p;
}

constexpr uint64_t kPrexPlanLimit = 1u << 16;  // larger plans: not eligible

// The threads (linear ids g) that decide a guarded input's verdict, or false.
bool prex_grid_plan(const Ir& ir, const cufz_input& in, uint32_t budget, std::vector<uint32_t>* out) {
  // shared loads are modelled as reading 0: true only while no loaded
  // shared value reaches a check
  if (!barriers_eliminable(ir)) return false;
  bool merged[3];
  for (int d = 0; d < 3; d++) merged[d] = true;
  for (int pass = 0; pass < 4; pass++) {
    PrexGrid pg{ir, in, budget, {merged[0], merged[1], merged[2]}};
    for (int d = 0; d < 3; d++) {
      pg.n[d] = in.block[d];
      pg.g[d] = in.grid[d];
    }
    PrexGrid::State st;
    st.r.assign(std::max(ir.n_regs, 1), PrexGrid::uni(0));
    if (!pg.exec(0, (int)ir.ops.size(), st)) {
      bool again = false;
      for (int d = 0; d < 3; d++)
        if (pg.need_split[d] && merged[d]) {
          merged[d] = false;
          again = true;
        }
      if (again) continue;
      return false;
    }
    // per dimension: the (t, b) pairs of the plan
    std::vector<std::pair<int64_t, int64_t>> tb[3];
    uint64_t total = 1;
    for (int d = 0; d < 3; d++) {
      if (merged[d]) {
        for (int64_t x : axis_points(pg.cut_g[d], pg.n[d] * pg.g[d]))
          tb[d].push_back({x % pg.n[d], x / pg.n[d]});
      } else {
        const std::vector<int64_t> pt = axis_points(pg.cut_t[d], pg.n[d]);
        const std::vector<int64_t> pb = axis_points(pg.cut_b[d], pg.g[d]);
        for (int64_t b : pb)
          for (int64_t t : pt) tb[d].push_back({t, b});
      }
      total *= tb[d].size();
      if (total > kPrexPlanLimit) return false;
    }
    const uint64_t T = (uint64_t)in.block[0] * in.block[1] * in.block[2];
    out->clear();
    for (const auto& z : tb[2])
      for (const auto& y : tb[1])
        for (const auto& x : tb[0]) {
          const uint64_t bl = x.second + (uint64_t)in.grid[0] * (y.second + (uint64_t)in.grid[1] * z.second);
          const uint64_t tl = x.first + (uint64_t)in.block[0] * (y.first + (uint64_t)in.block[1] * z.first);
          out->push_back((uint32_t)(bl * T + tl));
        }
    std::sort(out->begin(), out->end());
    out->erase(std::unique(out->begin(), out->end()), out->end());
    return true;
  }
  return false;
}

bool prex_run(const Ir& ir, const cufz_input& in, uint32_t budget) {
  if (!barriers_eliminable(ir)) return false;  // as in prex_grid_plan
  PrexRun run{ir, in, budget, {}, std::vector<AVal>(std::max(ir.n_regs, 1))};
  for (int d = 0; d < 3; d++) {
    run.ext[d] = (int64_t)in.block[d] - 1;
    run.ext[3 + d] = (int64_t)in.grid[d] - 1;
  }
  return run.exec(0, (int)ir.ops.size());
}

}  // namespace

// Launches the engine runs at all: valid shapes of at most 2^31 threads
// (their linear thread ids fit 32 bits).
bool prex_launch_ok(const cufz_input& in) {
  return !launch_rejected(in) && launch_within(in, 1ull << 31, nullptr);
}

bool prex_input_ok(const PrexInfo& p, const cufz_input& in, uint32_t iter_budget) {
  return prex_launch_ok(in) && prex_run(p.ir, in, iter_budget);
}

std::vector<uint32_t> prex_corners(const cufz_input& in) {
  std::vector<uint32_t> t[3], b[3];
  for (int d = 0; d < 3; d++) {
    t[d] = {0u};
    if (in.block[d] > 1) t[d].push_back(in.block[d] - 1);
    b[d] = {0u};
    if (in.grid[d] > 1) b[d].push_back(in.grid[d] - 1);
  }
  const uint64_t T = (uint64_t)in.block[0] * in.block[1] * in.block[2];
  std::vector<uint32_t> out;
  for (uint32_t bz : b[2])
    for (uint32_t by : b[1])
      for (uint32_t bx : b[0])
        for (uint32_t tz : t[2])
          for (uint32_t ty : t[1])
            for (uint32_t tx : t[0]) {
              const uint64_t bl = bx + (uint64_t)in.grid[0] * (by + (uint64_t)in.grid[1] * bz);
              const uint64_t tl = tx + (uint64_t)in.block[0] * (ty + (uint64_t)in.block[1] * tz);
              out.push_back((uint32_t)(bl * T + tl));
            }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
  return out;
}

bool prex_plan(const PrexInfo& p, const cufz_input& in, uint32_t iter_budget,
               std::vector<uint32_t>* threads) {
  if (!prex_launch_ok(in)) return false;
  if (prex_run(p.ir, in, iter_budget)) {
    *threads = prex_corners(in);
    return true;
  }
  return prex_grid_plan(p.ir, in, iter_budget, threads);
}

}  // namespace cufz

using namespace cufz;

extern "C" cufz_status cufz_prex_check(const void* bytes, size_t nbytes, const cufz_input* in,
                                       uint32_t iter_budget, uint32_t* eligible) {
  if (!bytes || !in || !eligible) return CUFZ_E_INVALID_ARG;
  PrexInfo p;
  if (!decode((const uint8_t*)bytes, nbytes, &p.ir)) return CUFZ_E_INVALID_PROGRAM;
  *eligible = prex_input_ok(p, *in, iter_budget ? iter_budget : 4096u) ? 1u : 0u;
  return CUFZ_OK;
}

extern "C" cufz_status cufz_prex_plan(const void* bytes, size_t nbytes, const cufz_input* in,
                                      uint32_t iter_budget, uint32_t* threads, uint32_t cap,
                                      uint32_t* n_threads) {
  if (!bytes || !in || !n_threads || (!threads && cap)) return CUFZ_E_INVALID_ARG;
  PrexInfo p;
  if (!decode((const uint8_t*)bytes, nbytes, &p.ir)) return CUFZ_E_INVALID_PROGRAM;
  std::vector<uint32_t> g;
  *n_threads = 0;
  if (!prex_plan(p, *in, iter_budget ? iter_budget : 4096u, &g)) return CUFZ_OK;
  *n_threads = (uint32_t)g.size();
  if (g.size() > cap) return CUFZ_E_NOMEM;
  std::copy(g.begin(), g.end(), threads);
  return CUFZ_OK;
}

