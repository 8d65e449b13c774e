// Host side of the batched ROS4 chemistry integrator: spec reader, mechanism compiler
// (per-mechanism CUDA source -> NVRTC -> sm_103a cubin), module cache and the C ABI of
// include/chem.h.  No torch types: callers pass device pointers and a cudaStream_t as void*.
#include "chem.h"

#include <cuda.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "device_src.inc"  // const char* const kDeviceSource: ros4_device.cuh as a string

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[2048];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CU_TRY(call)                                                               \
  do {                                                                             \
    CUresult _r = (call);                                                          \
    if (_r != CUDA_SUCCESS) {                                                      \
      const char* _s = nullptr;                                                    \
      drv::cuGetErrorString(_r, &_s);                                                   \
      return fail(CHEM_ECUDA, "%s failed: %s", #call, _s ? _s : "unknown error"); \
    }                                                                              \
  } while (0)


// ------------------------------------------------------------------------------ driver API
// The CUDA driver library is opened at run time so that this library loads (and can compile
// kernels with NVRTC) on machines without a GPU driver; any device call then fails cleanly.
namespace drv {
#define CHEM_STR2(x) #x
#define CHEM_STR(x) CHEM_STR2(x)
#define CHEM_DRV_FUNCS(X)                                                                       \
  X(cuInit) X(cuGetErrorString) X(cuCtxGetCurrent) X(cuCtxSetCurrent) X(cuCtxGetDevice)          \
  X(cuDeviceGet) X(cuDevicePrimaryCtxRetain) X(cuDeviceGetAttribute) X(cuModuleLoadData)        \
  X(cuModuleUnload) X(cuModuleGetFunction) X(cuModuleGetGlobal) X(cuFuncSetAttribute)           \
  X(cuFuncGetAttribute) X(cuOccupancyMaxActiveBlocksPerMultiprocessor) X(cuLaunchKernel)         \
  X(cuMemsetD32Async) X(cuMemcpyDtoH) X(cuMemcpyDtoHAsync) X(cuMemcpyHtoDAsync)                 \
  X(cuStreamSynchronize) X(cuMemHostAlloc) X(cuMemFreeHost) X(cuMemAlloc) X(cuMemFree)            \
  X(cuEventCreate) X(cuEventRecord) X(cuEventSynchronize) X(cuEventElapsedTime) X(cuEventDestroy) \
  X(cuMemcpyDtoDAsync)
#define CHEM_DECL(fn) decltype(&::fn) fn = nullptr;
CHEM_DRV_FUNCS(CHEM_DECL)
#undef CHEM_DECL
std::once_flag once;
std::string load_error;

bool load() {
  std::call_once(once, [] {
    void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
    if (!h) {
      load_error = std::string("cannot load the CUDA driver: ") + dlerror();
      return;
    }
#define CHEM_LOAD(fn)                                                   \
    fn = reinterpret_cast<decltype(fn)>(dlsym(h, CHEM_STR(fn)));        \
    if (!fn && load_error.empty()) load_error = "missing driver symbol " CHEM_STR(fn);
    CHEM_DRV_FUNCS(CHEM_LOAD)
#undef CHEM_LOAD
  });
  return load_error.empty();
}
}  // namespace drv

// ------------------------------------------------------------------------------ mechanism data

constexpr int kMaxSide = 3;  // distinct species per reaction side
constexpr size_t kSegLen = 8;  // entries per omega-gather segment

struct SpeciesData {
  std::string name;
  double W = 0;
  double Tmid = 1000;
  double nasa[2][7] = {};  // [low, high][a1..a7]
};

struct ReactionData {
  int kind = 0;  // 0 ELEM, 1 THIRD, 2 LIND, 3 TROE
  int nre = 0, npr = 0;
  int rsp[kMaxSide] = {}, rnu[kMaxSide] = {}, psp[kMaxSide] = {}, pnu[kMaxSide] = {};
  double lnA = 0, b = 0, theta = 0;  // SI
  std::vector<std::pair<int, double>> eff;  // non-default third-body efficiencies
  double lnA0 = 0, b0 = 0, theta0 = 0;
  double troe[4] = {};  // a, T***, T*, T**
};

struct MechData {
  std::string name;
  int n_elements = 0;
  std::vector<SpeciesData> sp;
  std::vector<ReactionData> rx;
};

// Spec reader (format documented in paper_2205_05681_gb300/synth.py).
struct LineReader {
  std::ifstream in;
  int lineno = 0;
  std::vector<std::string> tok;
  bool next() {
    std::string s;
    while (std::getline(in, s)) {
      ++lineno;
      const size_t h = s.find('#');
      if (h != std::string::npos) s.resize(h);
      tok.clear();
      std::istringstream ss(s);
      std::string t;
      while (ss >> t) tok.push_back(t);
      if (!tok.empty()) return true;
    }
    return false;
  }
};

bool to_double(const std::string& s, double* v) {
  char* end = nullptr;
  *v = std::strtod(s.c_str(), &end);
  return end && *end == '\0';
}
bool to_int(const std::string& s, int* v) {
  char* end = nullptr;
  long x = std::strtol(s.c_str(), &end, 10);
  *v = (int)x;
  return end && *end == '\0';
}

constexpr double kRcal = 1.987204258640832;  // cal/(mol K)
constexpr double kCgsToSi = 1e-3;            // cm^3/mol -> m^3/kmol

int read_spec(const char* path, MechData* m) {
  LineReader r;
  r.in.open(path);
  if (!r.in) return fail(CHEM_EIO, "cannot open spec file %s", path);
  std::map<std::string, int> idx;
  int want_sp = -1, want_rx = -1;
  auto bad = [&](const char* what) { return fail(CHEM_EIO, "%s:%d: %s", path, r.lineno, what); };
  auto side = [&](size_t& p, int* sp, int* nu, int* n) -> int {
    int cnt;
    if (p >= r.tok.size() || !to_int(r.tok[p++], &cnt) || cnt < 0 || cnt > kMaxSide) return -1;
    *n = cnt;
    for (int i = 0; i < cnt; ++i) {
      if (p + 1 >= r.tok.size()) return -1;
      auto it = idx.find(r.tok[p++]);
      if (it == idx.end()) return -1;
      sp[i] = it->second;
      if (!to_int(r.tok[p++], &nu[i]) || nu[i] < 1 || nu[i] > 3) return -1;
    }
    return 0;
  };
  while (r.next()) {
    const std::string& tag = r.tok[0];
    if (tag == "MECHANISM") {
      if (r.tok.size() > 1) m->name = r.tok[1];
    } else if (tag == "ELEMENTS") {
      m->n_elements = (int)r.tok.size() - 1;
    } else if (tag == "SPECIES") {
      if (r.tok.size() != 2 || !to_int(r.tok[1], &want_sp)) return bad("bad SPECIES line");
    } else if (tag == "SP") {
      const size_t need = 2 + 1 + m->n_elements + 5;
      if (r.tok.size() != need) return bad("bad SP line");
      SpeciesData s;
      s.name = r.tok[1];
      if (!to_double(r.tok[2], &s.W) || !(s.W > 0)) return bad("bad molecular weight");
      if (!to_double(r.tok[3 + m->n_elements + 1], &s.Tmid)) return bad("bad Tmid");
      idx[s.name] = (int)m->sp.size();
      m->sp.push_back(s);
    } else if (tag == "LO" || tag == "HI") {
      if (m->sp.empty() || r.tok.size() != 8) return bad("bad NASA line");
      double* a = m->sp.back().nasa[tag == "LO" ? 0 : 1];
      for (int i = 0; i < 7; ++i)
        if (!to_double(r.tok[1 + i], &a[i])) return bad("bad NASA coefficient");
    } else if (tag == "REACTIONS") {
      if (r.tok.size() != 2 || !to_int(r.tok[1], &want_rx)) return bad("bad REACTIONS line");
    } else if (tag == "R") {
      if (r.tok.size() < 2) return bad("bad R line");
      ReactionData x;
      const std::string& k = r.tok[1];
      x.kind = k == "ELEM" ? 0 : k == "THIRD" ? 1 : k == "LIND" ? 2 : k == "TROE" ? 3 : -1;
      if (x.kind < 0) return bad("unknown reaction type");
      size_t p = 2;
      if (side(p, x.rsp, x.rnu, &x.nre) || side(p, x.psp, x.pnu, &x.npr)) return bad("bad reaction side");
      if (x.nre == 0 || x.npr == 0) return bad("empty reaction side");
      double A, Ea;
      if (p + 3 != r.tok.size() || !to_double(r.tok[p], &A) || !to_double(r.tok[p + 1], &x.b) ||
          !to_double(r.tok[p + 2], &Ea) || !(A > 0))
        return bad("bad Arrhenius data");
      int order = (x.kind == 1) ? 1 : 0;
      for (int i = 0; i < x.nre; ++i) order += x.rnu[i];
      x.lnA = std::log(A) + (order - 1) * std::log(kCgsToSi);
      x.theta = Ea / kRcal;
      m->rx.push_back(x);
    } else if (tag == "EFF") {
      if (m->rx.empty()) return bad("EFF before R");
      int cnt;
      if (r.tok.size() < 2 || !to_int(r.tok[1], &cnt) || r.tok.size() != (size_t)(2 + 2 * cnt))
        return bad("bad EFF line");
      for (int i = 0; i < cnt; ++i) {
        auto it = idx.find(r.tok[2 + 2 * i]);
        double e;
        if (it == idx.end() || !to_double(r.tok[3 + 2 * i], &e)) return bad("bad efficiency");
        m->rx.back().eff.push_back({it->second, e});
      }
    } else if (tag == "LOW") {
      if (m->rx.empty() || r.tok.size() != 4) return bad("bad LOW line");
      ReactionData& x = m->rx.back();
      double A0, Ea0;
      if (!to_double(r.tok[1], &A0) || !to_double(r.tok[2], &x.b0) || !to_double(r.tok[3], &Ea0) || !(A0 > 0))
        return bad("bad LOW data");
      int order = 1;
      for (int i = 0; i < x.nre; ++i) order += x.rnu[i];
      x.lnA0 = std::log(A0) + (order - 1) * std::log(kCgsToSi);
      x.theta0 = Ea0 / kRcal;
    } else if (tag == "TROE") {
      if (m->rx.empty() || r.tok.size() != 5) return bad("bad TROE line");
      for (int i = 0; i < 4; ++i)
        if (!to_double(r.tok[1 + i], &m->rx.back().troe[i])) return bad("bad TROE data");
    } else if (tag == "END") {
      break;
    } else {
      return bad("unknown record");
    }
  }
  if ((int)m->sp.size() != want_sp || (int)m->rx.size() != want_rx)
    return fail(CHEM_EIO, "%s: species/reaction counts do not match the declared counts", path);
  if (m->sp.size() < 2) return fail(CHEM_EIO, "%s: need at least two species", path);
  for (auto& x : m->rx) {
    if (x.kind >= 2 && x.lnA0 == 0 && x.b0 == 0) return fail(CHEM_EIO, "%s: falloff reaction without LOW", path);
    if (x.kind == 3 && !(x.troe[1] > 0 && x.troe[2] > 0)) return fail(CHEM_EIO, "%s: bad TROE temperatures", path);
  }
  return 0;
}

// ------------------------------------------------------------------------------ code generation

// The Rosenbrock methods of the paper's solver table, in transformed variables (gamma, a_ij,
// c_ij, m_i, error weights e_i), entered from their publications:
//   0 ROS4   Hairer & Wanner, Solving ODEs II, Sec. IV.7 (L-stable, order 4(3)) -- the default;
//   1 ROS3   Sandu et al. (1997), order 3(2), L-stable;
//   2 RODAS3 Sandu et al. (1997), order 3(2), stiffly accurate;
//   3 RODAS4 Hairer & Wanner, Sec. VI.4, order 4(3), stiffly accurate;
//   5 ROS2   Verwer et al. (1999), a W-method of order 2(1), used with Jacobian reuse.
struct RosCoefficients {
  int s = 0, order = 0;
  double gamma = 0;
  double a[6][6] = {}, c[6][6] = {}, m[6] = {}, e[6] = {};
  bool erk = false;  // explicit Runge-Kutta in increment form u_i = h f(y + sum a_ij u_j)
};

RosCoefficients ros_coefficients(int id) {
  RosCoefficients t;
  if (id == 5) {
    // ROS2 (Verwer, Spee, Blom & Hundsdorfer 1999): second order for any matrix in place of the
    // Jacobian (a W-method), L-stable with g = 1 + 1/sqrt(2); transformed: a21 = 1/g,
    // c21 = -2/g, m = (3/(2g), 1/(2g)), error weights (1/(2g), 1/(2g))
    t.s = 2; t.order = 2; t.gamma = 1.0 + 1.0 / std::sqrt(2.0);
    const double g = t.gamma;
    t.a[1][0] = 1.0 / g;
    t.c[1][0] = -2.0 / g;
    t.m[0] = 1.5 / g; t.m[1] = 0.5 / g;
    t.e[0] = 0.5 / g; t.e[1] = 0.5 / g;
    return t;
  }
  if (id == 4) {
    // Runge-Kutta-Fehlberg 4(5): the fifth-order weights are propagated, their difference to the
    // fourth-order ones is the error estimate (controller exponent 1/5)
    t.s = 6; t.order = 5; t.erk = true;
    t.a[1][0] = 1.0 / 4.0;
    t.a[2][0] = 3.0 / 32.0; t.a[2][1] = 9.0 / 32.0;
    t.a[3][0] = 1932.0 / 2197.0; t.a[3][1] = -7200.0 / 2197.0; t.a[3][2] = 7296.0 / 2197.0;
    t.a[4][0] = 439.0 / 216.0; t.a[4][1] = -8.0; t.a[4][2] = 3680.0 / 513.0; t.a[4][3] = -845.0 / 4104.0;
    t.a[5][0] = -8.0 / 27.0; t.a[5][1] = 2.0; t.a[5][2] = -3544.0 / 2565.0; t.a[5][3] = 1859.0 / 4104.0;
    t.a[5][4] = -11.0 / 40.0;
    const double b5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
    const double b4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
    for (int i = 0; i < 6; ++i) { t.m[i] = b5[i]; t.e[i] = b5[i] - b4[i]; }
    return t;
  }
  if (id == 1) {
    t.s = 3; t.order = 3; t.gamma = 0.43586652150845899941601945119356;
    t.a[1][0] = 1.0; t.a[2][0] = 1.0;
    t.c[1][0] = -1.0156171083877702091975600115545;
    t.c[2][0] = 4.0759956452537699824805835358067; t.c[2][1] = 9.2076794298330791242156818474003;
    t.m[0] = 1.0; t.m[1] = 6.1697947043828245592553615689730; t.m[2] = -0.42772256543218573326238373806514;
    t.e[0] = 0.5; t.e[1] = -2.9079558716805469821718236208017; t.e[2] = 0.22354069897811569627360909276199;
  } else if (id == 2) {
    t.s = 4; t.order = 3; t.gamma = 0.5;
    t.a[2][0] = 2.0; t.a[3][0] = 2.0; t.a[3][2] = 1.0;
    t.c[1][0] = 4.0; t.c[2][0] = 1.0; t.c[2][1] = -1.0; t.c[3][0] = 1.0; t.c[3][1] = -1.0; t.c[3][2] = -8.0 / 3.0;
    t.m[0] = 2.0; t.m[2] = 1.0; t.m[3] = 1.0;
    t.e[3] = 1.0;
  } else if (id == 3) {
    t.s = 6; t.order = 4; t.gamma = 0.25;
    const double a5[4] = {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.6878860361058950};
    t.a[1][0] = 1.544;
    t.a[2][0] = 0.9466785280815826; t.a[2][1] = 0.2557011698983284;
    t.a[3][0] = 3.314825187068521; t.a[3][1] = 2.896124015972201; t.a[3][2] = 0.9986419139977817;
    for (int j = 0; j < 4; ++j) { t.a[4][j] = a5[j]; t.a[5][j] = a5[j]; t.m[j] = a5[j]; }
    t.a[5][4] = 1.0;
    t.c[1][0] = -5.6688;
    t.c[2][0] = -2.430093356833875; t.c[2][1] = -0.2063599157091915;
    t.c[3][0] = -0.1073529058151375; t.c[3][1] = -9.594562251023355; t.c[3][2] = -20.47028614809616;
    t.c[4][0] = 7.496443313967647; t.c[4][1] = -10.24680431464352; t.c[4][2] = -33.99990352819905;
    t.c[4][3] = 11.70890893206160;
    t.c[5][0] = 8.083246795921522; t.c[5][1] = -7.981132988064893; t.c[5][2] = -31.52159432874371;
    t.c[5][3] = 16.31930543123136; t.c[5][4] = -6.058818238834054;
    t.m[4] = 1.0; t.m[5] = 1.0;
    t.e[5] = 1.0;
  } else {
    t.s = 4; t.order = 4; t.gamma = 0.57282;
    t.a[1][0] = 2.0;
    t.a[2][0] = 1.867943637803922; t.a[2][1] = 0.2344449711399156;
    t.a[3][0] = 1.867943637803922; t.a[3][1] = 0.2344449711399156;
    t.c[1][0] = -7.137615036412310;
    t.c[2][0] = 2.580708087951457; t.c[2][1] = 0.6515950076447975;
    t.c[3][0] = -2.137148994382534; t.c[3][1] = -0.3214669691237626; t.c[3][2] = -0.6949742501781779;
    t.m[0] = 2.255570073418735; t.m[1] = 0.2870493262186792; t.m[2] = 0.4353179431840180; t.m[3] = 1.093502252409163;
    t.e[0] = -0.2815431932141155; t.e[1] = -0.07276199124938920; t.e[2] = -0.1082196201495311;
    t.e[3] = -1.093502252409163;
  }
  return t;
}

// per stage: 1 = f at a new argument, 0 = the previous stage's argument again, 2 = the argument is y
std::vector<int> stage_f_reuse(const RosCoefficients& t) {
  std::vector<int> nf(t.s, 1);
  for (int i = 1; i < t.s; ++i) {
    bool zero = true, same = i > 1;
    for (int j = 0; j < 6; ++j) {
      zero = zero && t.a[i][j] == 0.0;
      if (i > 1) same = same && t.a[i][j] == t.a[i - 1][j];
    }
    nf[i] = zero ? 2 : (same ? 0 : 1);
  }
  return nf;
}

bool needs_f0(const RosCoefficients& t) {
  for (int v : stage_f_reuse(t)) if (v == 2) return true;
  return false;
}

std::string num(double v) {
  char b[40];
  snprintf(b, sizeof(b), "%.17g", v);
  std::string s(b);
  if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
  return s;
}

template <class F>
void emit_array(std::ostringstream& o, const char* type, const char* name, const std::string& dims, int n, F f) {
  o << "__device__ const " << type << " " << name << dims << " = {";
  for (int i = 0; i < n; ++i) o << (i ? "," : "") << f(i);
  o << "};\n";
}

// Kernel order of the reactions: grouped by the branches the reaction code takes (kind, Troe
// T** term, third-body efficiency count, reactant and product counts and coefficients), stable
// within a group.  Lanes of a warp take consecutive reactions, so grouped reactions keep the
// warp on one path (mechanisms that interleave falloff and plain reactions would otherwise pay
// the falloff branch in almost every warp).  costliest_first puts the falloff groups first, so
// that they fill whole warps while the last, partly filled round of the team's loop takes
// elementary reactions (a warp instruction costs its FP64 pipe time whatever the number of its
// active lanes): the forward modules take it (+5% at 53 species); the adjoint module keeps the
// cheapest groups first, with which its reverse sweep measured 9% faster (GB300, 53 species).
// Returns order[kernel index] = mechanism index.
std::vector<int> kernel_reaction_order(const MechData& m, bool costliest_first) {
  std::vector<int> order(m.rx.size());
  for (size_t r = 0; r < order.size(); ++r) order[r] = (int)r;
  auto key = [&](int r) {
    const ReactionData& x = m.rx[r];
    int neff = 0;
    if (x.kind != 0)
      for (auto& e : x.eff) neff += e.second != 1.0;
    std::vector<int> k = {x.kind, x.kind == 3 && x.troe[3] > 0.0, neff, x.nre, x.npr};
    for (int i = 0; i < x.nre; ++i) k.push_back(x.rnu[i]);
    for (int i = 0; i < x.npr; ++i) k.push_back(x.pnu[i]);
    return k;
  };
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return costliest_first ? key(b) < key(a) : key(a) < key(b); });
  return order;
}

std::string emit_mechanism(const MechData& m0, int team, int tpb, bool adjoint, int tableau) {
  const std::vector<int> order = kernel_reaction_order(m0, !adjoint);
  MechData m = m0;
  for (size_t r = 0; r < order.size(); ++r) m.rx[r] = m0.rx[order[r]];
  const int ns = (int)m.sp.size(), nr = (int)m.rx.size();
  std::ostringstream o;
  o << "// generated for mechanism " << m.name << "\n";
  if (adjoint) o << "#define CHEM_ADJOINT 1\n#define CHEM_ADJ_SCRATCH_BYTES " << CHEM_ADJ_SCRATCH_BYTES << "\n";
  o << "#define NS " << ns << "\n#define NR " << nr << "\n#define TEAM " << team << "\n#define TPB " << tpb
    << "\n#define MAXP " << kMaxSide << "\n";
  const RosCoefficients c = ros_coefficients(tableau);
  const std::vector<int> nf = stage_f_reuse(c);
  o << "#define TABLEAU_ID " << tableau << "\n#define ERK " << (c.erk ? 1 : 0) << "\n#define RS " << c.s
    << "\n#define RORDER " << c.order
    << "\n#define NEED_F0 " << (needs_f0(c) ? 1 : 0) << "\n#define RGAM " << num(c.gamma) << "\n";
  emit_array(o, "double", "rk_a", "[" + std::to_string(c.s * c.s) + "]", c.s * c.s,
             [&](int i) { return num(c.a[i / c.s][i % c.s]); });
  emit_array(o, "double", "rk_c", "[" + std::to_string(c.s * c.s) + "]", c.s * c.s,
             [&](int i) { return num(c.c[i / c.s][i % c.s]); });
  emit_array(o, "double", "rk_m", "[" + std::to_string(c.s) + "]", c.s, [&](int i) { return num(c.m[i]); });
  emit_array(o, "double", "rk_e", "[" + std::to_string(c.s) + "]", c.s, [&](int i) { return num(c.e[i]); });
  emit_array(o, "int", "rk_newf", "[" + std::to_string(c.s) + "]", c.s, [&](int i) { return std::to_string(nf[i]); });
  if (tableau == 0) {  // named ROS4 coefficients used by the adjoint
    o << "#define RA21 " << num(c.a[1][0]) << "\n#define RA31 " << num(c.a[2][0]) << "\n#define RA32 " << num(c.a[2][1])
      << "\n#define RC21 " << num(c.c[1][0]) << "\n#define RC31 " << num(c.c[2][0]) << "\n#define RC32 " << num(c.c[2][1])
      << "\n#define RC41 " << num(c.c[3][0]) << "\n#define RC42 " << num(c.c[3][1]) << "\n#define RC43 " << num(c.c[3][2])
      << "\n#define RM1 " << num(c.m[0]) << "\n#define RM2 " << num(c.m[1]) << "\n#define RM3 " << num(c.m[2])
      << "\n#define RM4 " << num(c.m[3]) << "\n";
  }
  const double Wb = m.sp[ns - 1].W;
  emit_array(o, "double", "mk_W", "[" + std::to_string(ns) + "]", ns, [&](int k) { return num(m.sp[k].W); });
  emit_array(o, "double", "mk_invW", "[" + std::to_string(ns) + "]", ns, [&](int k) { return num(1.0 / m.sp[k].W); });
  emit_array(o, "double", "mk_wratio", "[" + std::to_string(std::max(ns - 1, 1)) + "]", ns - 1,
             [&](int k) { return num(m.sp[k].W / Wb); });
  emit_array(o, "double", "mk_Tmid", "[" + std::to_string(ns) + "]", ns, [&](int k) { return num(m.sp[k].Tmid); });
  // NASA-7 with the divisions folded: cp/R (a1..a5), h/RT (a1, a2/2, a3/3, a4/4, a5/5, a6),
  // s/R (a1 [x lnT], a2, a3/2, a4/3, a5/4, -, a7), dcp/dT/R (a2, 2a3, 3a4, 4a5)
  auto nasa_table = [&](const char* name, int width, std::function<double(const double*, int)> f) {
    o << "__device__ const double " << name << "[" << ns << "][2][" << width << "] = {";
    for (int k = 0; k < ns; ++k) {
      o << (k ? "," : "") << "{";
      for (int r = 0; r < 2; ++r) {
        o << (r ? "," : "") << "{";
        for (int i = 0; i < width; ++i) o << (i ? "," : "") << num(f(m.sp[k].nasa[r], i));
        o << "}";
      }
      o << "}";
    }
    o << "};\n";
  };
  nasa_table("mk_cp", 5, [](const double* a, int i) { return a[i]; });
  nasa_table("mk_h", 6, [](const double* a, int i) { return i < 5 ? a[i] / (i + 1) : a[5]; });
  nasa_table("mk_s", 7, [](const double* a, int i) {
    if (i == 0) return a[0];
    if (i < 5) return a[i] / i;
    return i == 6 ? a[6] : 0.0;
  });
  nasa_table("mk_dcp", 4, [](const double* a, int i) { return a[i + 1] * (i + 1); });
  const std::string R = "[" + std::to_string(nr) + "]";
  const std::string RP = "[" + std::to_string(nr) + "][" + std::to_string(kMaxSide) + "]";
  emit_array(o, "int", "mk_rorig", R, nr, [&](int r) { return std::to_string(order[r]); });
  emit_array(o, "int", "mk_kind", R, nr, [&](int r) { return std::to_string(m.rx[r].kind); });
  emit_array(o, "double", "mk_lnA", R, nr, [&](int r) { return num(m.rx[r].lnA); });
  emit_array(o, "double", "mk_b", R, nr, [&](int r) { return num(m.rx[r].b); });
  emit_array(o, "double", "mk_th", R, nr, [&](int r) { return num(m.rx[r].theta); });
  emit_array(o, "int", "mk_nre", R, nr, [&](int r) { return std::to_string(m.rx[r].nre); });
  emit_array(o, "int", "mk_npr", R, nr, [&](int r) { return std::to_string(m.rx[r].npr); });
  auto side_table = [&](const char* name, int ReactionData::*cnt, int (ReactionData::*arr)[kMaxSide]) {
    o << "__device__ const int " << name << RP << " = {";
    for (int r = 0; r < nr; ++r) {
      o << (r ? "," : "") << "{";
      for (int i = 0; i < kMaxSide; ++i) o << (i ? "," : "") << (i < m.rx[r].*cnt ? (m.rx[r].*arr)[i] : 0);
      o << "}";
    }
    o << "};\n";
  };
  side_table("mk_rsp", &ReactionData::nre, &ReactionData::rsp);
  side_table("mk_rnu", &ReactionData::nre, &ReactionData::rnu);
  side_table("mk_psp", &ReactionData::npr, &ReactionData::psp);
  side_table("mk_pnu", &ReactionData::npr, &ReactionData::pnu);
  emit_array(o, "int", "mk_dnu", R, nr, [&](int r) {
    int d = 0;
    for (int i = 0; i < m.rx[r].npr; ++i) d += m.rx[r].pnu[i];
    for (int i = 0; i < m.rx[r].nre; ++i) d -= m.rx[r].rnu[i];
    return std::to_string(d);
  });
  // the same coefficients as doubles: the rate arithmetic reads them without an integer-to-FP64
  // conversion (on GB300 every FP64-pipe instruction is scarce)
  auto side_table_f = [&](const char* name, int ReactionData::*cnt, int (ReactionData::*arr)[kMaxSide]) {
    o << "__device__ const double " << name << RP << " = {";
    for (int r = 0; r < nr; ++r) {
      o << (r ? "," : "") << "{";
      for (int i = 0; i < kMaxSide; ++i) o << (i ? "," : "") << (i < m.rx[r].*cnt ? (m.rx[r].*arr)[i] : 0) << ".0";
      o << "}";
    }
    o << "};\n";
  };
  side_table_f("mk_rnuf", &ReactionData::nre, &ReactionData::rnu);
  side_table_f("mk_pnuf", &ReactionData::npr, &ReactionData::pnu);
  emit_array(o, "double", "mk_dnuf", R, nr, [&](int r) {
    int d = 0;
    for (int i = 0; i < m.rx[r].npr; ++i) d += m.rx[r].pnu[i];
    for (int i = 0; i < m.rx[r].nre; ++i) d -= m.rx[r].rnu[i];
    return std::to_string(d) + ".0";
  });
  std::vector<int> off(nr + 1, 0), esp;
  std::vector<double> eval;
  for (int r = 0; r < nr; ++r) {
    off[r] = (int)esp.size();
    if (m.rx[r].kind != 0)
      for (auto& e : m.rx[r].eff)
        if (e.second != 1.0) { esp.push_back(e.first); eval.push_back(e.second - 1.0); }
  }
  off[nr] = (int)esp.size();
  const int ne = std::max<int>(1, (int)esp.size());
  emit_array(o, "int", "mk_effoff", "[" + std::to_string(nr + 1) + "]", nr + 1, [&](int i) { return std::to_string(off[i]); });
  emit_array(o, "int", "mk_effsp", "[" + std::to_string(ne) + "]", ne,
             [&](int i) { return std::to_string(i < (int)esp.size() ? esp[i] : 0); });
  emit_array(o, "double", "mk_effval", "[" + std::to_string(ne) + "]", ne,
             [&](int i) { return num(i < (int)eval.size() ? eval[i] : 0.0); });
  emit_array(o, "double", "mk_lnA0", R, nr, [&](int r) { return num(m.rx[r].lnA0); });
  emit_array(o, "double", "mk_b0", R, nr, [&](int r) { return num(m.rx[r].b0); });
  emit_array(o, "double", "mk_th0", R, nr, [&](int r) { return num(m.rx[r].theta0); });
  o << "__device__ const double mk_troe[" << nr << "][4] = {";
  for (int r = 0; r < nr; ++r) {
    const double* t = m.rx[r].troe;
    const bool tr = m.rx[r].kind == 3;
    o << (r ? "," : "") << "{" << num(tr ? t[0] : 0.0) << "," << num(tr ? 1.0 / t[1] : 0.0) << ","
      << num(tr ? 1.0 / t[2] : 0.0) << "," << num(tr ? t[3] : 0.0) << "}";
  }
  o << "};\n";
  // species -> (reaction, net nu) lists cut into segments of at most kSegLen entries for the
  // deterministic omega gather of multi-lane teams
  std::vector<int> gbeg(1, 0), grx, spseg(1, 0);
  std::vector<double> gnu;
  for (int k = 0; k < ns; ++k) {
    std::vector<std::pair<int, int>> lst;
    for (int r = 0; r < nr; ++r) {
      int nu = 0;
      for (int i = 0; i < m.rx[r].npr; ++i) if (m.rx[r].psp[i] == k) nu += m.rx[r].pnu[i];
      for (int i = 0; i < m.rx[r].nre; ++i) if (m.rx[r].rsp[i] == k) nu -= m.rx[r].rnu[i];
      if (nu) lst.push_back({r, nu});
    }
    for (size_t a = 0; a < lst.size(); a += kSegLen) {
      for (size_t b = a; b < std::min(lst.size(), a + kSegLen); ++b) { grx.push_back(lst[b].first); gnu.push_back(lst[b].second); }
      gbeg.push_back((int)grx.size());
    }
    spseg.push_back((int)gbeg.size() - 1);
  }
  const int nseg = (int)gbeg.size() - 1, nent = std::max<int>(1, (int)grx.size());
  o << "#define NSEG " << std::max(nseg, 1) << "\n";
  emit_array(o, "int", "mk_gseg_beg", "[" + std::to_string(nseg + 1) + "]", nseg + 1, [&](int i) { return std::to_string(gbeg[i]); });
  emit_array(o, "int", "mk_gent_rx", "[" + std::to_string(nent) + "]", nent,
             [&](int i) { return std::to_string(i < (int)grx.size() ? grx[i] : 0); });
  emit_array(o, "double", "mk_gent_nu", "[" + std::to_string(nent) + "]", nent,
             [&](int i) { return num(i < (int)gnu.size() ? gnu[i] : 0.0); });
  emit_array(o, "int", "mk_spseg_beg", "[" + std::to_string(ns + 1) + "]", ns + 1, [&](int i) { return std::to_string(spseg[i]); });
  o << kDeviceSource;
  o << "\nextern \"C\" __device__ const int chem_slots = SLOTS;\n";
  o << "extern \"C\" __device__ const int chem_tstride = TSTRIDE;\n";
  return o.str();
}

// ------------------------------------------------------------------------------ NVRTC + cache

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ULL) {
  for (unsigned char c : s) { h ^= c; h *= 1099511628211ULL; }
  return h;
}

const std::vector<std::string> kNvrtcOptions = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo",
                                                "--ptxas-options=-v", "-DNDEBUG"};

int nvrtc_compile(const std::string& src, const std::string& name, std::string* cubin, std::string* log,
                  const std::vector<std::string>& name_exprs = {}, std::vector<std::string>* lowered = nullptr) {
  nvrtcProgram prog;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), name.c_str(), 0, nullptr, nullptr);
  if (r != NVRTC_SUCCESS) return fail(CHEM_ENVRTC, "nvrtcCreateProgram: %s", nvrtcGetErrorString(r));
  for (auto& e : name_exprs) nvrtcAddNameExpression(prog, e.c_str());
  std::vector<const char*> opts;
  for (auto& s : kNvrtcOptions) opts.push_back(s.c_str());
  r = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  size_t logsz = 0;
  nvrtcGetProgramLogSize(prog, &logsz);
  std::string lg(logsz, '\0');
  if (logsz) nvrtcGetProgramLog(prog, &lg[0]);
  if (log) *log = lg;
  if (r != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return fail(CHEM_ENVRTC, "NVRTC compile of %s failed: %s\n%s", name.c_str(), nvrtcGetErrorString(r),
                lg.substr(0, 1500).c_str());
  }
  if (lowered) {
    lowered->clear();
    for (auto& e : name_exprs) {
      const char* low = nullptr;
      if (nvrtcGetLoweredName(prog, e.c_str(), &low) != NVRTC_SUCCESS || !low) {
        nvrtcDestroyProgram(&prog);
        return fail(CHEM_ENVRTC, "no lowered name for %s", e.c_str());
      }
      lowered->push_back(low);
    }
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  cubin->resize(n);
  nvrtcGetCUBIN(prog, &(*cubin)[0]);
  nvrtcDestroyProgram(&prog);
  return 0;
}

// The adjoint module's static scratch array (used by chem_adjoint_noalloc only): the name
// expression that keeps it in the module, and its lowered (internal-linkage) symbol name, which
// is checked against NVRTC's whenever the module is compiled.
const char* const kAdjScratchExpr = "&chem_adj_scratch";
const char* const kAdjScratchSym = "chem_adj_scratch";

// cubin for (mechanism, team, block): from cache_dir if present, else compiled (and stored)
int build_cubin(const MechData& m, int team, int tpb, bool adjoint, int tableau, const char* cache_dir, bool verbose,
                std::string* cubin, std::string* log) {
  const std::string src = emit_mechanism(m, team, tpb, adjoint, tableau);
  int major = 0, minor = 0;
  nvrtcVersion(&major, &minor);
  std::string key = src;
  for (auto& s : kNvrtcOptions) key += "|" + s;
  key += "|nvrtc" + std::to_string(major) + "." + std::to_string(minor);
  char hex[32];
  snprintf(hex, sizeof(hex), "%016llx", (unsigned long long)fnv1a(key));
  std::string path;
  if (cache_dir && *cache_dir) {
    path = std::string(cache_dir) + "/" + m.name + (adjoint ? "_adj" : "") + "_r" + std::to_string(tableau) + "_t" +
           std::to_string(team) + "_b" + std::to_string(tpb) + "_" + hex + ".cubin";
    std::ifstream in(path, std::ios::binary);
    if (in) {
      std::ostringstream ss;
      ss << in.rdbuf();
      *cubin = ss.str();
      if (!cubin->empty()) return 0;
    }
  }
  std::string lg;
  std::vector<std::string> exprs, lowered;
  if (adjoint) exprs.push_back(kAdjScratchExpr);
  int rc = nvrtc_compile(src, m.name + ".cu", cubin, &lg, exprs, &lowered);
  if (!rc && adjoint && lowered[0] != kAdjScratchSym)
    return fail(CHEM_ENVRTC, "unexpected lowered name %s for the adjoint scratch", lowered[0].c_str());
  if (log) *log = lg;
  if (verbose && !lg.empty()) fprintf(stderr, "[chem] %s team=%d block=%d\n%s\n", m.name.c_str(), team, tpb, lg.c_str());
  if (rc) return rc;
  if (!path.empty()) {
    const std::string tmp = path + ".tmp" + std::to_string((long long)std::hash<std::string>{}(hex));
    std::ofstream out(tmp, std::ios::binary);
    out.write(cubin->data(), (std::streamsize)cubin->size());
    out.close();
    if (out) std::rename(tmp.c_str(), path.c_str());
  }
  return 0;
}

// ------------------------------------------------------------------------------ modules

struct Module {
  int team = 0, tpb = 0;
  CUmodule mod = nullptr;
  CUfunction f_source = nullptr, f_jac = nullptr, f_int = nullptr, f_pinit = nullptr, f_patt = nullptr,
             f_pfin = nullptr, f_adj = nullptr, f_adjred = nullptr, f_vjp = nullptr, f_ohist = nullptr,
             f_oscan = nullptr, f_oscat = nullptr, f_route = nullptr, f_rfall = nullptr;
  int smem = 0;          // dynamic shared memory per block
  int adj_smem = 0;      // ... of the adjoint / VJP kernels (0: not available for this config)
  int adj_occ = 0;
  CUdeviceptr adj_scratch = 0;   // device address of the adjoint module's static scratch array
  size_t adj_scratch_bytes = 0;
  int occ = 0;           // resident blocks per SM for f_int
  int regs = 0;
};

}  // namespace

struct chem_mech {
  MechData data;
  std::string cache_dir;
  bool verbose = false;
  CUcontext ctx = nullptr;
  int n_sm = 0;
  int default_team = 32, default_tpb = 64;
  std::mutex mu;       // guards modules
  std::mutex host_mu;  // guards the chem_integrate_host buffers
  // keyed by (lanes per cell, threads per block, Rosenbrock method)
  std::map<std::tuple<int, int, int>, std::unique_ptr<Module>> modules;      // forward kernels
  std::map<std::tuple<int, int, int>, std::unique_ptr<Module>> adj_modules;  // + adjoint kernels
  // plain-mode host mirror of the activity counter and host-API buffers
  unsigned int* pinned = nullptr;
  CUdeviceptr host_api_buf = 0;
  size_t host_api_bytes = 0;
};

namespace {

// shared-memory slots of one cell; mirrors the OFF_* layout of ros4_device.cuh: A, Y, U1, YT,
// U2..Us, [F0], six per-species arrays, the packed permutation (and pivots with one lane per
// cell), 24 reduction slots
int slots_for(const MechData& m, int tableau, int team) {
  const int ns = (int)m.sp.size();
  const RosCoefficients c = ros_coefficients(tableau);
  const int packed = (ns + 1) / 2;
  // stage slots: at least three after the stage argument (the Jacobian assembly aliases them)
  return ns * ns + (8 + std::max(c.s, 3) + (needs_f0(c) ? 1 : 0)) * ns + packed * (team == 1 ? 2 : 1) + 24;
}

// distance in doubles between consecutive teams' slots (TSTRIDE of ros4_device.cuh): sub-warp
// teams pad to TEAM (mod 16) so that the teams of a half-warp hit disjoint banks
int tstride_for(const MechData& m, int tableau, int team) {
  const int sl = slots_for(m, tableau, team);
  if (team > 1 && team < 32) return sl + ((team - sl % 16 + 16) % 16);
  return sl;
}

// default kernel configuration by mechanism size (the autotuner's usual pick on GB300):
// two warps per cell up to 64 species, eight warps per cell above
void default_config(int ns, int* team, int* tpb) {
  if (ns <= 64) { *team = 64; *tpb = 64; }
  else { *team = 256; *tpb = 256; }
}

int check_config(int team, int tpb) {
  if (team == 1 && (tpb == 32 || tpb == 64 || tpb == 128)) return 0;
  if ((team == 4 || team == 8 || team == 16) && (tpb == 32 || tpb == 64 || tpb == 128)) return 0;
  if (team == 32 && tpb % 32 == 0 && tpb >= 32 && tpb <= 256) return 0;
  if ((team == 64 || team == 128 || team == 256) && tpb == team) return 0;
  return fail(CHEM_EARG, "unsupported kernel config team=%d block=%d", team, tpb);
}

int smem_bytes(const MechData& m, int team, int tpb, int tableau) {
  const int teams = team <= 32 ? tpb / team : 1;
  return tstride_for(m, tableau, team) * 8 * teams;
}

int get_module(chem_mech* m, int team, int tpb, Module** out, bool adjoint = false, int tableau = 0,
               const std::string* prebuilt = nullptr) {
  std::lock_guard<std::mutex> lk(m->mu);
  if (tableau < 0 || tableau > 5) return fail(CHEM_EARG, "unknown integration method %d", tableau);
  auto key = std::make_tuple(team, tpb, tableau);
  auto& mods = adjoint ? m->adj_modules : m->modules;
  auto it = mods.find(key);
  if (it != mods.end()) { *out = it->second.get(); return 0; }
  if (int rc = check_config(team, tpb)) return rc;
  const int smem = smem_bytes(m->data, team, tpb, tableau);
  int max_optin = 0;
  CUdevice dev;
  CU_TRY(drv::cuCtxGetDevice(&dev));
  CU_TRY(drv::cuDeviceGetAttribute(&max_optin, CU_DEVICE_ATTRIBUTE_MAX_SHARED_MEMORY_PER_BLOCK_OPTIN, dev));
  if (smem > max_optin)
    return fail(CHEM_EARG, "config team=%d block=%d needs %d B shared memory (max %d)", team, tpb, smem, max_optin);
  std::string cubin, log;
  if (prebuilt && !prebuilt->empty()) cubin = *prebuilt;
  else if (int rc = build_cubin(m->data, team, tpb, adjoint, tableau, m->cache_dir.c_str(), m->verbose, &cubin, &log))
    return rc;
  auto mod = std::make_unique<Module>();
  mod->team = team;
  mod->tpb = tpb;
  mod->smem = smem;
  CU_TRY(drv::cuModuleLoadData(&mod->mod, cubin.data()));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_source, mod->mod, "chem_eval_source_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_jac, mod->mod, "chem_eval_jacobian_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_int, mod->mod, "chem_integrate_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_pinit, mod->mod, "chem_plain_init_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_patt, mod->mod, "chem_plain_attempt_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_pfin, mod->mod, "chem_plain_finish_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_ohist, mod->mod, "chem_order_hist_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_oscan, mod->mod, "chem_order_scan_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_oscat, mod->mod, "chem_order_scatter_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_route, mod->mod, "chem_route_k"));
  CU_TRY(drv::cuModuleGetFunction(&mod->f_rfall, mod->mod, "chem_route_fallback_k"));
  CUdeviceptr slots_ptr;
  size_t slots_sz;
  CU_TRY(drv::cuModuleGetGlobal(&slots_ptr, &slots_sz, mod->mod, "chem_slots"));
  int dev_slots = 0;
  CU_TRY(drv::cuMemcpyDtoH(&dev_slots, slots_ptr, sizeof(int)));
  if (dev_slots != slots_for(m->data, tableau, team))
    return fail(CHEM_ECUDA, "shared-memory layout mismatch (%d vs %d)", dev_slots,
                slots_for(m->data, tableau, team));
  CU_TRY(drv::cuModuleGetGlobal(&slots_ptr, &slots_sz, mod->mod, "chem_tstride"));
  CU_TRY(drv::cuMemcpyDtoH(&dev_slots, slots_ptr, sizeof(int)));
  if (dev_slots != tstride_for(m->data, tableau, team))
    return fail(CHEM_ECUDA, "team stride mismatch (%d vs %d)", dev_slots, tstride_for(m->data, tableau, team));
  for (CUfunction f : {mod->f_source, mod->f_jac, mod->f_int, mod->f_pinit, mod->f_patt}) {
    CU_TRY(drv::cuFuncSetAttribute(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, smem));
    // all of L1 as shared memory: occupancy is bounded by the cells' shared-memory footprint
    CU_TRY(drv::cuFuncSetAttribute(f, CU_FUNC_ATTRIBUTE_PREFERRED_SHARED_MEMORY_CARVEOUT, 100));
  }
  CU_TRY(drv::cuOccupancyMaxActiveBlocksPerMultiprocessor(&mod->occ, mod->f_int, tpb, smem));
  if (adjoint && team >= 32) {
    CUdeviceptr ap;
    size_t asz;
    CU_TRY(drv::cuModuleGetGlobal(&ap, &asz, mod->mod, "chem_aslots"));
    int aslots = 0;
    CU_TRY(drv::cuMemcpyDtoH(&aslots, ap, sizeof(int)));
    const int asmem = aslots * 8 * (team <= 32 ? tpb / team : 1);
    if (asmem <= max_optin) {
      CU_TRY(drv::cuModuleGetFunction(&mod->f_adj, mod->mod, "chem_adjoint_k"));
      CU_TRY(drv::cuModuleGetFunction(&mod->f_adjred, mod->mod, "chem_adjoint_reduce_k"));
      CU_TRY(drv::cuModuleGetFunction(&mod->f_vjp, mod->mod, "chem_eval_vjp_k"));
      CU_TRY(drv::cuFuncSetAttribute(mod->f_adj, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, asmem));
      CU_TRY(drv::cuFuncSetAttribute(mod->f_adj, CU_FUNC_ATTRIBUTE_PREFERRED_SHARED_MEMORY_CARVEOUT, 100));
      CU_TRY(drv::cuFuncSetAttribute(mod->f_vjp, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, asmem));
      CU_TRY(drv::cuOccupancyMaxActiveBlocksPerMultiprocessor(&mod->adj_occ, mod->f_adj, tpb, asmem));
      if (mod->adj_occ >= 1) mod->adj_smem = asmem;
    }
  }
  CU_TRY(drv::cuFuncGetAttribute(&mod->regs, CU_FUNC_ATTRIBUTE_NUM_REGS, mod->f_int));
  if (mod->occ < 1) return fail(CHEM_ECUDA, "config team=%d block=%d cannot be resident", team, tpb);
  *out = mod.get();
  mods[key] = std::move(mod);
  return 0;
}

int resolve(chem_mech* m, const chem_int_opts* o, Module** mod) {
  int team = m->default_team, tpb = m->default_tpb;
  if (o && o->team > 0) {
    team = o->team;
    tpb = o->block > 0 ? o->block : (team <= 32 ? 64 : team);
  }
  return get_module(m, team, tpb, mod, false, o ? o->tableau : 0);
}

int make_current(chem_mech* m) {
  CU_TRY(drv::cuCtxSetCurrent(m->ctx));
  return 0;
}

int teams_per_block(const Module* mod) { return mod->team <= 32 ? mod->tpb / mod->team : 1; }

unsigned grid_for(const chem_mech* m, const Module* mod, int64_t n_cells) {
  const int64_t tpb = teams_per_block(mod);
  const int64_t need = (n_cells + tpb - 1) / tpb;
  const int64_t cap = (int64_t)m->n_sm * mod->occ;
  return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

int launch(CUfunction f, unsigned grid, const Module* mod, void* stream, void** args) {
  CU_TRY(drv::cuLaunchKernel(f, grid, 1, 1, mod->tpb, 1, 1, mod->smem, (CUstream)stream, args, nullptr));
  return 0;
}

int check_cells(int64_t n, int64_t ld) {
  if (n < 0) return fail(CHEM_EARG, "n_cells < 0");
  if (ld < n) return fail(CHEM_EARG, "ld (%lld) < n_cells (%lld)", (long long)ld, (long long)n);
  return 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PlainLayout {
  size_t y, t, h, flags, att, st, cnt, total;
};

PlainLayout plain_layout(int ns, int64_t n, int max_steps) {
  PlainLayout L;
  size_t o = 0;
  L.y = o; o = align256(o + sizeof(double) * ns * n);
  L.t = o; o = align256(o + sizeof(double) * n);
  L.h = o; o = align256(o + sizeof(double) * n);
  L.flags = o; o = align256(o + sizeof(int) * n);
  L.att = o; o = align256(o + sizeof(int) * n);
  L.st = o; o = align256(o + sizeof(int) * n);
  L.cnt = o; o = align256(o + sizeof(unsigned) * ((size_t)max_steps + 2));
  L.total = o;
  return L;
}

}  // namespace

// ================================================================================ C ABI

extern "C" {

const char* chem_last_error(void) { return g_last_error.c_str(); }

int chem_mech_compile_only(const char* spec_path, const chem_build_opts* opts, char* log, size_t log_cap) {
  if (!spec_path) return fail(CHEM_EARG, "spec_path is NULL");
  MechData d;
  if (int rc = read_spec(spec_path, &d)) return rc;
  int team, tpb;
  default_config((int)d.sp.size(), &team, &tpb);
  if (opts && opts->team > 0) { team = opts->team; tpb = opts->block > 0 ? opts->block : tpb; }
  if (int rc = check_config(team, tpb)) return rc;
  std::string cubin, lg;
  const bool adj = opts && opts->adjoint;
  if (adj && team < 32) return fail(CHEM_EARG, "the adjoint needs a multi-lane configuration (team >= 32)");
  const int tab = opts ? opts->tableau : 0;
  if (tab < 0 || tab > 5) return fail(CHEM_EARG, "unknown integration method %d", tab);
  if (adj && tab != 0) return fail(CHEM_EARG, "the adjoint is implemented for ROS4 (tableau 0)");
  int rc = build_cubin(d, team, tpb, adj, tab, opts ? opts->cache_dir : nullptr, opts && opts->verbose, &cubin, &lg);
  if (log && log_cap) {
    const size_t n = std::min(lg.size(), log_cap - 1);
    memcpy(log, lg.data(), n);
    log[n] = '\0';
  }
  return rc;
}

int chem_mech_load(const char* spec_path, const chem_build_opts* opts, chem_mech_t* out) {
  if (!spec_path || !out) return fail(CHEM_EARG, "NULL argument");
  *out = nullptr;
  auto m = std::make_unique<chem_mech>();
  if (int rc = read_spec(spec_path, &m->data)) return rc;
  if (opts && opts->cache_dir) m->cache_dir = opts->cache_dir;
  m->verbose = opts && opts->verbose;
  if (!drv::load()) return fail(CHEM_ECUDA, "%s", drv::load_error.c_str());
  CU_TRY(drv::cuInit(0));
  CUcontext ctx = nullptr;
  CU_TRY(drv::cuCtxGetCurrent(&ctx));
  if (!ctx) {
    CUdevice dev;
    CU_TRY(drv::cuDeviceGet(&dev, 0));
    CU_TRY(drv::cuDevicePrimaryCtxRetain(&ctx, dev));
    CU_TRY(drv::cuCtxSetCurrent(ctx));
  }
  m->ctx = ctx;
  CUdevice dev;
  CU_TRY(drv::cuCtxGetDevice(&dev));
  CU_TRY(drv::cuDeviceGetAttribute(&m->n_sm, CU_DEVICE_ATTRIBUTE_MULTIPROCESSOR_COUNT, dev));
  default_config((int)m->data.sp.size(), &m->default_team, &m->default_tpb);
  if (opts && opts->team > 0) {
    m->default_team = opts->team;
    m->default_tpb = opts->block > 0 ? opts->block : m->default_tpb;
  }
  Module* mod;
  if (int rc = get_module(m.get(), m->default_team, m->default_tpb, &mod)) return rc;
  CU_TRY(drv::cuMemHostAlloc((void**)&m->pinned, 64 * sizeof(unsigned), 0));
  *out = m.release();
  return 0;
}

int chem_mech_free(chem_mech_t m) {
  if (!m) return 0;
  drv::cuCtxSetCurrent(m->ctx);
  for (auto& kv : m->modules) drv::cuModuleUnload(kv.second->mod);
  for (auto& kv : m->adj_modules) drv::cuModuleUnload(kv.second->mod);
  if (m->pinned) drv::cuMemFreeHost(m->pinned);
  if (m->host_api_buf) drv::cuMemFree(m->host_api_buf);
  delete m;
  return 0;
}

int chem_mech_info(chem_mech_t m, int32_t* ns, int32_t* nr, int32_t* ne) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (ns) *ns = (int32_t)m->data.sp.size();
  if (nr) *nr = (int32_t)m->data.rx.size();
  if (ne) *ne = m->data.n_elements;
  return 0;
}

int chem_mech_lnA(chem_mech_t m, double* lnA) {
  if (!m || !lnA) return fail(CHEM_EARG, "NULL argument");
  for (size_t r = 0; r < m->data.rx.size(); ++r) lnA[r] = m->data.rx[r].lnA;
  return 0;
}

static int eval_common(chem_mech_t m, bool jac, int64_t n_cells, const double* T, const double* P,
                       const double* n, double* out, int64_t ld, const double* lnA, void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = check_cells(n_cells, ld)) return rc;
  if (n_cells == 0) return 0;
  if (!T || !P || !n || !out) return fail(CHEM_EARG, "NULL array");
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = resolve(m, nullptr, &mod)) return rc;
  long long nc = n_cells, l = ld;
  void* args[] = {&nc, (void*)&T, (void*)&P, (void*)&n, &out, &l, (void*)&lnA};
  return launch(jac ? mod->f_jac : mod->f_source, grid_for(m, mod, n_cells), mod, stream, args);
}

int chem_eval_source(chem_mech_t m, int64_t n_cells, const double* T, const double* P, const double* n, double* f,
                     int64_t ld, const double* lnA, void* stream) {
  return eval_common(m, false, n_cells, T, P, n, f, ld, lnA, stream);
}

int chem_eval_jacobian(chem_mech_t m, int64_t n_cells, const double* T, const double* P, const double* n, double* J,
                       int64_t ld, const double* lnA, void* stream) {
  return eval_common(m, true, n_cells, T, P, n, J, ld, lnA, stream);
}

size_t chem_integrate_workspace(chem_mech_t m, int64_t n_cells, const chem_int_opts* o) {
  if (!m || n_cells < 0) return 0;
  const int mode = o ? o->mode : CHEM_MODE_PERSISTENT;
  if (mode == CHEM_MODE_PLAIN) {
    const int max_steps = (o && o->max_steps > 0) ? o->max_steps : 100000;
    return plain_layout((int)m->data.sp.size(), n_cells, max_steps).total;
  }
  if (o && o->cell_method)  // two queue counters, list lengths, two cell lists, explicit status
    return 512 + 3 * align256(sizeof(int) * (size_t)n_cells);
  return 256;
}

int chem_kernel_config(chem_mech_t m, const chem_int_opts* o, int32_t* team, int32_t* block, int32_t* smem,
                       int32_t* regs) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = resolve(m, o, &mod)) return rc;
  if (team) *team = mod->team;
  if (block) *block = mod->tpb;
  if (smem) *smem = mod->smem;
  if (regs) *regs = mod->regs;
  return 0;
}

int chem_integrate(chem_mech_t m, int64_t n_cells, double* T, const double* P, double* Y, int64_t ld, double dt,
                   double rtol, double atol, double* h, int32_t* status, const chem_int_opts* o, void* ws,
                   size_t ws_bytes, void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = check_cells(n_cells, ld)) return rc;
  if (!(dt > 0) || !(rtol > 0) || !(atol > 0) || !std::isfinite(dt))
    return fail(CHEM_EARG, "dt, rtol and atol must be positive and finite");
  if (n_cells == 0) return 0;
  if (!T || !P || !Y) return fail(CHEM_EARG, "NULL array");
  const int mode = o ? o->mode : CHEM_MODE_PERSISTENT;
  int max_steps = (o && o->max_steps > 0) ? o->max_steps : 100000;
  double h_min = (o && o->h_min > 0) ? o->h_min : 1e-20;
  double T_min = o ? o->T_min : 0.0;
  const double* lnA = o ? o->lnA : nullptr;
  int* att = o ? o->attempts : nullptr;
  const size_t need = chem_integrate_workspace(m, n_cells, o);
  if (!ws || ws_bytes < need) return fail(CHEM_EWS, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if (((uintptr_t)ws) & 255) return fail(CHEM_EARG, "workspace must be 256-byte aligned");
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = resolve(m, o, &mod)) return rc;
  long long nc = n_cells, l = ld;
  CUstream s = (CUstream)stream;
  double* wjc = o ? o->jac_cache : nullptr;  // W-method factorisation cache
  const int alt = (o && o->alt_tableau) ? o->alt_tableau : 4;
  if (wjc && !(o->tableau == 5 || (o->cell_method && alt == 5)))
    return fail(CHEM_EARG, "jac_cache needs the W-method (tableau 5, or alt_tableau 5 with cell_method)");
  if (wjc && mode != CHEM_MODE_PERSISTENT) return fail(CHEM_EARG, "jac_cache needs the persistent driver");
  if (wjc && (((uintptr_t)wjc) & 7)) return fail(CHEM_EARG, "jac_cache must be 8-byte aligned");
  if (mode == CHEM_MODE_PERSISTENT && o && o->cell_method) {
    // per-cell method switching: route, explicit launch, fall back, implicit launch
    if (o->tableau < 0 || o->tableau > 3)
      return fail(CHEM_EARG, "per-cell method switching needs a Rosenbrock method (tableau 0..3)");
    if (alt != 4 && alt != 5) return fail(CHEM_EARG, "alt_tableau must be CHEM_RKF45 or CHEM_ROS2W");
    if (alt == 5 && !wjc) return fail(CHEM_EARG, "switching to the W-method needs jac_cache");
    Module* emod;
    if (int rc = get_module(m, mod->team, mod->tpb, &emod, false, alt)) return rc;
    char* b = (char*)ws;
    const CUdeviceptr qe = (CUdeviceptr)b, qi = (CUdeviceptr)(b + 64);
    unsigned* counts = (unsigned*)(b + 256);
    const size_t li = align256(sizeof(int) * (size_t)n_cells);
    int* list_e = (int*)(b + 512);
    int* list_i = (int*)(b + 512 + li);
    int* st_e = (int*)(b + 512 + 2 * li);
    int* cm = o->cell_method;
    CU_TRY(drv::cuMemsetD32Async((CUdeviceptr)counts, 0, 2, s));
    CU_TRY(drv::cuMemsetD32Async(qe, 0, 2, s));
    CU_TRY(drv::cuMemsetD32Async(qi, 0, 2, s));
    const unsigned g256 = (unsigned)((n_cells + 255) / 256);
    {
      void* a[] = {&nc, &cm, &list_e, &list_i, &counts};
      CU_TRY(drv::cuLaunchKernel(mod->f_route, g256, 1, 1, 256, 1, 1, 0, s, a, nullptr));
    }
    int* tnacc = nullptr;
    double* th = nullptr;
    double* tck = nullptr;
    int cap = 0, interval = 1;
    {
      CUdeviceptr q = qe;
      const unsigned* cnt = counts;
      int keep = 1, am = 1;
      void* a[] = {&nc, &T, (void*)&P, &Y, &l, &dt, &rtol, &atol, &h, &st_e, &att, (void*)&lnA,
                   &max_steps, &h_min, &T_min, &q, &tnacc, &th, &tck, &cap, &interval, &list_e,
                   (void*)&cnt, &keep, &cm, &am, &wjc};
      if (int rc = launch(emod->f_int, grid_for(m, emod, n_cells), emod, stream, a)) return rc;
    }
    {
      void* a[] = {&nc, &list_e, &counts, &st_e, &list_i, &status};
      CU_TRY(drv::cuLaunchKernel(mod->f_rfall, g256, 1, 1, 256, 1, 1, 0, s, a, nullptr));
    }
    CUdeviceptr q = qi;
    const unsigned* cnt = counts + 1;
    int keep = 0, am = alt == 5 ? 3 : 2;
    void* a[] = {&nc, &T, (void*)&P, &Y, &l, &dt, &rtol, &atol, &h, &status, &att, (void*)&lnA,
                 &max_steps, &h_min, &T_min, &q, &tnacc, &th, &tck, &cap, &interval, &list_i,
                 (void*)&cnt, &keep, &cm, &am, &wjc};
    return launch(mod->f_int, grid_for(m, mod, n_cells), mod, stream, a);
  }
  if (mode == CHEM_MODE_PERSISTENT) {
    CUdeviceptr q = (CUdeviceptr)ws;
    CU_TRY(drv::cuMemsetD32Async(q, 0, 2, s));
    int* tnacc = nullptr;
    double* th = nullptr;
    double* tck = nullptr;
    int cap = 0, interval = 1, keep = 0;
    const int32_t* order = o ? o->order : nullptr;
    const unsigned* ocount = nullptr;
    int* cm = nullptr;
    int am = 0;
    void* args[] = {&nc, &T, (void*)&P, &Y, &l, &dt, &rtol, &atol, &h, &status, &att, (void*)&lnA,
                    &max_steps, &h_min, &T_min, &q, &tnacc, &th, &tck, &cap, &interval,
                    (void*)&order, (void*)&ocount, &keep, &cm, &am, &wjc};
    return launch(mod->f_int, grid_for(m, mod, n_cells), mod, stream, args);
  }
  if (mode != CHEM_MODE_PLAIN) return fail(CHEM_EARG, "unknown mode %d", mode);
  // plain driver: init, then one launch per attempt until no cell is active
  const int ns = (int)m->data.sp.size();
  PlainLayout L = plain_layout(ns, n_cells, max_steps);
  char* base = (char*)ws;
  double* wy = (double*)(base + L.y);
  double* wt = (double*)(base + L.t);
  double* wh = (double*)(base + L.h);
  int* wfl = (int*)(base + L.flags);
  int* wat = (int*)(base + L.att);
  int* wst = (int*)(base + L.st);
  unsigned* cnt = (unsigned*)(base + L.cnt);
  CU_TRY(drv::cuMemsetD32Async((CUdeviceptr)cnt, 0, (size_t)max_steps + 2, s));
  const unsigned grid = grid_for(m, mod, n_cells);
  {
    void* args[] = {&nc, &T, &Y, &l, &dt, (void*)&h, &T_min, &wy, &wt, &wh, &wfl, &wat, &wst};
    if (int rc = launch(mod->f_pinit, grid, mod, stream, args)) return rc;
  }
  {
    void* args[] = {&nc, &status, &att, &wst, &wfl};
    CU_TRY(drv::cuLaunchKernel(mod->f_pfin, (unsigned)((n_cells + 255) / 256), 1, 1, 256, 1, 1, 0, s, args, nullptr));
  }
  // the attempt counter of every active cell grows by one per launch, so max_steps + 1
  // launches retire every cell; the host checks the activity counter every few launches
  const int poll = 4;
  for (int it = 0; it <= max_steps; ++it) {
    unsigned* c = cnt + it;
    void* args[] = {&nc, &T, (void*)&P, &Y, &l, &dt, &rtol, &atol, &h, &status, &att, (void*)&lnA,
                    &max_steps, &h_min, &wy, &wt, &wh, &wfl, &wat, &wst, &c};
    if (int rc = launch(mod->f_patt, grid, mod, stream, args)) return rc;
    if (it % poll == poll - 1 || it == max_steps) {
      CU_TRY(drv::cuMemcpyDtoHAsync(m->pinned, (CUdeviceptr)c, sizeof(unsigned), s));
      CU_TRY(drv::cuStreamSynchronize(s));
      if (m->pinned[0] == 0) break;
    }
  }
  return 0;
}

int chem_integrate_host(chem_mech_t m, int64_t n_cells, double* T, const double* P, double* Y, double dt, double rtol,
                        double atol, double* h, int32_t* status, const chem_int_opts* o, void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (n_cells <= 0) return n_cells == 0 ? 0 : fail(CHEM_EARG, "n_cells < 0");
  if (!T || !P || !Y) return fail(CHEM_EARG, "NULL array");
  if (int rc = make_current(m)) return rc;
  const int ns = (int)m->data.sp.size();
  chem_int_opts oo = o ? *o : chem_int_opts{};
  oo.mode = CHEM_MODE_PERSISTENT;
  oo.attempts = nullptr;
  oo.order = nullptr;
  oo.cell_method = nullptr;
  oo.jac_cache = nullptr;
  const size_t n = (size_t)n_cells;
  const size_t offT = 0, offP = align256(offT + 8 * n), offY = align256(offP + 8 * n),
               offH = align256(offY + 8 * n * ns), offS = align256(offH + 8 * n), offW = align256(offS + 4 * n);
  const size_t total = offW + 256;
  std::lock_guard<std::mutex> lk(m->host_mu);
  if (m->host_api_bytes < total) {
    if (m->host_api_buf) CU_TRY(drv::cuMemFree(m->host_api_buf));
    m->host_api_buf = 0;
    m->host_api_bytes = 0;
    CU_TRY(drv::cuMemAlloc(&m->host_api_buf, total));
    m->host_api_bytes = total;
  }
  CUstream s = (CUstream)stream;
  const CUdeviceptr b = m->host_api_buf;
  CU_TRY(drv::cuMemcpyHtoDAsync(b + offT, T, 8 * n, s));
  CU_TRY(drv::cuMemcpyHtoDAsync(b + offP, P, 8 * n, s));
  CU_TRY(drv::cuMemcpyHtoDAsync(b + offY, Y, 8 * n * ns, s));
  if (h) CU_TRY(drv::cuMemcpyHtoDAsync(b + offH, h, 8 * n, s));
  int rc = chem_integrate(m, n_cells, (double*)(b + offT), (const double*)(b + offP), (double*)(b + offY), n_cells,
                          dt, rtol, atol, h ? (double*)(b + offH) : nullptr, status ? (int32_t*)(b + offS) : nullptr,
                          &oo, (void*)(b + offW), 256, stream);
  if (rc) return rc;
  CU_TRY(drv::cuMemcpyDtoHAsync(T, b + offT, 8 * n, s));
  CU_TRY(drv::cuMemcpyDtoHAsync(Y, b + offY, 8 * n * ns, s));
  if (h) CU_TRY(drv::cuMemcpyDtoHAsync(h, b + offH, 8 * n, s));
  if (status) CU_TRY(drv::cuMemcpyDtoHAsync(status, b + offS, 4 * n, s));
  CU_TRY(drv::cuStreamSynchronize(s));
  return 0;
}

// ------------------------------------------------------------------------------ adjoint

static size_t tape_ck_count(int cap, int interval) { return (size_t)((cap - 1) / interval + 1); }

struct TapeLayout {
  size_t nacc, h, ck, total;
};

static TapeLayout tape_layout(int ns, int64_t n, int cap, int interval) {
  TapeLayout L;
  size_t o = 0;
  L.nacc = o; o = align256(o + sizeof(int) * n);
  L.h = o; o = align256(o + sizeof(double) * n * (size_t)cap);
  L.ck = o; o = align256(o + sizeof(double) * n * ns * tape_ck_count(cap, interval));
  L.total = o;
  return L;
}

size_t chem_tape_bytes(chem_mech_t m, int64_t n_cells, int32_t capacity, int32_t interval) {
  if (!m || n_cells < 0 || capacity < 1 || interval < 1) return 0;
  return tape_layout((int)m->data.sp.size(), n_cells, capacity, interval).total;
}

static int check_tape(chem_mech_t m, int64_t n_cells, const chem_tape* t) {
  if (!t || !t->mem) return fail(CHEM_EARG, "NULL tape");
  if (t->n_cells != n_cells) return fail(CHEM_EARG, "tape was sized for %lld cells", (long long)t->n_cells);
  if (t->capacity < 1 || t->interval < 1) return fail(CHEM_EARG, "tape capacity and interval must be >= 1");
  if (t->bytes < chem_tape_bytes(m, n_cells, t->capacity, t->interval)) return fail(CHEM_EWS, "tape memory too small");
  if (((uintptr_t)t->mem) & 255) return fail(CHEM_EARG, "tape memory must be 256-byte aligned");
  return 0;
}

int chem_integrate_ckpt(chem_mech_t m, int64_t n_cells, double* T, const double* P, double* Y, int64_t ld, double dt,
                        double rtol, double atol, double* h, int32_t* status, const chem_int_opts* o,
                        const chem_tape* tape, void* ws, size_t ws_bytes, void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = check_cells(n_cells, ld)) return rc;
  if (!(dt > 0) || !(rtol > 0) || !(atol > 0) || !std::isfinite(dt))
    return fail(CHEM_EARG, "dt, rtol and atol must be positive and finite");
  if (n_cells == 0) return 0;
  if (!T || !P || !Y) return fail(CHEM_EARG, "NULL array");
  if (int rc = check_tape(m, n_cells, tape)) return rc;
  if (o && o->mode != CHEM_MODE_PERSISTENT) return fail(CHEM_EARG, "the checkpointed forward is persistent only");
  if (!ws || ws_bytes < 256 || (((uintptr_t)ws) & 255)) return fail(CHEM_EWS, "workspace of 256 aligned bytes needed");
  int max_steps = (o && o->max_steps > 0) ? o->max_steps : 100000;
  double h_min = (o && o->h_min > 0) ? o->h_min : 1e-20;
  double T_min = o ? o->T_min : 0.0;
  const double* lnA = o ? o->lnA : nullptr;
  int* att = o ? o->attempts : nullptr;
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = resolve(m, o, &mod)) return rc;
  const TapeLayout L = tape_layout((int)m->data.sp.size(), n_cells, tape->capacity, tape->interval);
  char* b = (char*)tape->mem;
  int* tnacc = (int*)(b + L.nacc);
  double* th = (double*)(b + L.h);
  double* tck = (double*)(b + L.ck);
  int cap = tape->capacity, interval = tape->interval;
  long long nc = n_cells, l = ld;
  CUdeviceptr q = (CUdeviceptr)ws;
  CU_TRY(drv::cuMemsetD32Async(q, 0, 2, (CUstream)stream));
  const int32_t* order = o ? o->order : nullptr;
  const unsigned* ocount = nullptr;
  int keep = 0;
  int* cm = nullptr;
  int am = 0;
  if (o && o->cell_method) return fail(CHEM_EARG, "the checkpointed forward has no per-cell method switching");
  double* wjc = nullptr;
  void* args[] = {&nc, &T, (void*)&P, &Y, &l, &dt, &rtol, &atol, &h, &status, &att, (void*)&lnA,
                  &max_steps, &h_min, &T_min, &q, &tnacc, &th, &tck, &cap, &interval, (void*)&order,
                  (void*)&ocount, &keep, &cm, &am, &wjc};
  return launch(mod->f_int, grid_for(m, mod, n_cells), mod, stream, args);
}

static int adjoint_module(chem_mech_t m, const chem_int_opts* o, Module** mod) {
  Module* fwd;
  if (o && o->tableau != 0) return fail(CHEM_EARG, "the adjoint is implemented for ROS4 (tableau 0)");
  if (int rc = resolve(m, o, &fwd)) return rc;
  if (fwd->team < 32) return fail(CHEM_EARG, "the adjoint needs a multi-lane configuration (team >= 32)");
  if (int rc = get_module(m, fwd->team, fwd->tpb, mod, true)) return rc;
  if (!(*mod)->f_adj)
    return fail(CHEM_EARG, "the adjoint needs a multi-lane configuration (team >= 32) that fits shared memory");
  return 0;
}

static int64_t adjoint_teams(const chem_mech* m, const Module* mod, int64_t n_cells) {
  const int64_t tpb = teams_per_block(mod);
  const int64_t need = (n_cells + tpb - 1) / tpb;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)m->n_sm * mod->adj_occ));
  return grid * tpb;
}

size_t chem_adjoint_workspace(chem_mech_t m, int64_t n_cells, const chem_int_opts* o, int32_t interval) {
  if (!m || n_cells < 0 || interval < 1) return 0;
  if (make_current(m)) return 0;
  Module* mod;
  if (adjoint_module(m, o, &mod)) return 0;
  const int ns = (int)m->data.sp.size(), nr = (int)m->data.rx.size();
  const int64_t teams = adjoint_teams(m, mod, std::max<int64_t>(n_cells, 1));
  return 256 + align256(sizeof(double) * teams * (size_t)interval * ns) + align256(sizeof(double) * teams * nr);
}

int chem_adjoint(chem_mech_t m, int64_t n_cells, const double* P, const double* gT, const double* gY, int64_t ld,
                 const chem_tape* tape, const chem_int_opts* o, double* g_lnA, double* gT0, double* gY0, void* ws,
                 size_t ws_bytes, void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = check_cells(n_cells, ld)) return rc;
  if (!P || !gT || !gY || !g_lnA || !gT0 || !gY0) return fail(CHEM_EARG, "NULL array");
  if (int rc = check_tape(m, n_cells, tape)) return rc;
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = adjoint_module(m, o, &mod)) return rc;
  const size_t need = chem_adjoint_workspace(m, n_cells, o, tape->interval);
  if (!ws || ws_bytes < need) return fail(CHEM_EWS, "adjoint workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if (((uintptr_t)ws) & 255) return fail(CHEM_EARG, "workspace must be 256-byte aligned");
  const int ns = (int)m->data.sp.size(), nr = (int)m->data.rx.size();
  CUstream s = (CUstream)stream;
  if (n_cells == 0) {
    CU_TRY(drv::cuMemsetD32Async((CUdeviceptr)g_lnA, 0, 2 * (size_t)nr, s));
    return 0;
  }
  const int64_t teams = adjoint_teams(m, mod, n_cells);
  char* b = (char*)ws;
  CUdeviceptr q = (CUdeviceptr)b;
  double* seg = (double*)(b + 256);
  double* part = (double*)(b + 256 + align256(sizeof(double) * teams * (size_t)tape->interval * ns));
  const TapeLayout L = tape_layout(ns, n_cells, tape->capacity, tape->interval);
  char* tb = (char*)tape->mem;
  const int* tnacc = (const int*)(tb + L.nacc);
  const double* th = (const double*)(tb + L.h);
  const double* tck = (const double*)(tb + L.ck);
  const double* lnA = o ? o->lnA : nullptr;
  int interval = tape->interval;
  long long nc = n_cells, l = ld, nparts = teams;
  CU_TRY(drv::cuMemsetD32Async(q, 0, 2, s));
  void* args[] = {&nc, (void*)&P, (void*)&gT, (void*)&gY, &l, &gT0, &gY0, (void*)&lnA, (void*)&tnacc, (void*)&th,
                  (void*)&tck, &interval, &seg, &part, &q};
  const unsigned grid = (unsigned)(teams / teams_per_block(mod));
  CU_TRY(drv::cuLaunchKernel(mod->f_adj, grid, 1, 1, mod->tpb, 1, 1, mod->adj_smem, s, args, nullptr));
  void* rargs[] = {&nparts, &part, &g_lnA};
  CU_TRY(drv::cuLaunchKernel(mod->f_adjred, (unsigned)((nr + 127) / 128), 1, 1, 128, 1, 1, 0, s, rargs, nullptr));
  return 0;
}

int chem_adjoint_noalloc(chem_mech_t m, int64_t n_cells, const double* P, const double* gT, const double* gY,
                         int64_t ld, const chem_tape* tape, const chem_int_opts* o, double* g_lnA, double* gT0,
                         double* gY0, void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = check_cells(n_cells, ld)) return rc;
  if (!P || !gT || !gY || !g_lnA || !gT0 || !gY0) return fail(CHEM_EARG, "NULL array");
  if (int rc = check_tape(m, n_cells, tape)) return rc;
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = adjoint_module(m, o, &mod)) return rc;
  {
    // set-up, once per loaded adjoint module (one per device context, made current above): the
    // device address of the module's static scratch array
    std::lock_guard<std::mutex> lk(m->mu);
    if (!mod->adj_scratch) {
      CUdeviceptr p = 0;
      size_t bytes = 0;
      CU_TRY(drv::cuModuleGetGlobal(&p, &bytes, mod->mod, kAdjScratchSym));
      if (bytes < (size_t)CHEM_ADJ_SCRATCH_BYTES)
        return fail(CHEM_ECUDA, "static adjoint scratch is %zu bytes, expected %d", bytes, (int)CHEM_ADJ_SCRATCH_BYTES);
      mod->adj_scratch_bytes = bytes;
      mod->adj_scratch = p;
    }
  }
  const int ns = (int)m->data.sp.size(), nr = (int)m->data.rx.size();
  CUstream s = (CUstream)stream;
  if (n_cells == 0) {
    CU_TRY(drv::cuMemsetD32Async((CUdeviceptr)g_lnA, 0, 2 * (size_t)nr, s));
    return 0;
  }
  // scratch: [queue counter: 256 B][segment states: teams x interval x Ns][partials: teams x Nr]
  const size_t per_team = sizeof(double) * ((size_t)tape->interval * ns + nr);
  const size_t room = (size_t)CHEM_ADJ_SCRATCH_BYTES - 512;
  const int64_t tpb = teams_per_block(mod);
  const int64_t fit_blocks = (int64_t)(room / (per_team * (size_t)tpb));
  if (fit_blocks < 1)
    return fail(CHEM_EWS,
                "chem_adjoint_noalloc: one block of %lld cells needs %zu bytes of scratch (interval %d x %d species + "
                "%d reactions per cell); the static scratch holds %d bytes -- lower the checkpoint interval or "
                "use chem_adjoint with a workspace",
                (long long)tpb, per_team * (size_t)tpb, tape->interval, ns, nr, (int)CHEM_ADJ_SCRATCH_BYTES);
  int64_t teams = adjoint_teams(m, mod, n_cells);
  teams = std::min<int64_t>(teams, fit_blocks * tpb);
  const CUdeviceptr base = mod->adj_scratch;
  CUdeviceptr q = base;
  double* seg = (double*)(base + 256);
  double* part = (double*)(base + 256 + align256(sizeof(double) * teams * (size_t)tape->interval * ns));
  const TapeLayout L = tape_layout(ns, n_cells, tape->capacity, tape->interval);
  char* tb = (char*)tape->mem;
  const int* tnacc = (const int*)(tb + L.nacc);
  const double* th = (const double*)(tb + L.h);
  const double* tck = (const double*)(tb + L.ck);
  const double* lnA = o ? o->lnA : nullptr;
  int interval = tape->interval;
  long long nc = n_cells, l = ld, nparts = teams;
  // the scratch keeps the previous call's contents: the queue counter must start at zero; the
  // segment states and the partial rows are written before they are read
  CU_TRY(drv::cuMemsetD32Async(q, 0, 2, s));
  void* args[] = {&nc, (void*)&P, (void*)&gT, (void*)&gY, &l, &gT0, &gY0, (void*)&lnA, (void*)&tnacc, (void*)&th,
                  (void*)&tck, &interval, &seg, &part, &q};
  CU_TRY(drv::cuLaunchKernel(mod->f_adj, (unsigned)(teams / tpb), 1, 1, mod->tpb, 1, 1, mod->adj_smem, s, args, nullptr));
  void* rargs[] = {&nparts, &part, &g_lnA};
  CU_TRY(drv::cuLaunchKernel(mod->f_adjred, (unsigned)((nr + 127) / 128), 1, 1, 128, 1, 1, 0, s, rargs, nullptr));
  return 0;
}

int chem_eval_vjp(chem_mech_t m, int64_t n_cells, const double* T, const double* P, const double* n, const double* v,
                  double* gy, double* gp, int64_t ld, const double* lnA, void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = check_cells(n_cells, ld)) return rc;
  if (n_cells == 0) return 0;
  if (!T || !P || !n || !v || !gy || !gp) return fail(CHEM_EARG, "NULL array");
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = adjoint_module(m, nullptr, &mod)) return rc;
  long long nc = n_cells, l = ld;
  void* args[] = {&nc, (void*)&T, (void*)&P, (void*)&n, (void*)&v, &gy, &gp, &l, (void*)&lnA};
  const int64_t tpb = teams_per_block(mod);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_cells + tpb - 1) / tpb, (int64_t)m->n_sm * mod->adj_occ));
  CU_TRY(drv::cuLaunchKernel(mod->f_vjp, grid, 1, 1, mod->tpb, 1, 1, mod->adj_smem, (CUstream)stream, args, nullptr));
  return 0;
}

size_t chem_jac_cache_bytes(chem_mech_t m, int64_t n_cells) {
  if (!m || n_cells < 0) return 0;
  const size_t ns = m->data.sp.size();
  const size_t stride = ns * ns + 2 * ((ns + 1) / 2) + 2;  // WC_STRIDE of ros4_device.cuh
  return sizeof(double) * stride * (size_t)n_cells;
}

size_t chem_cost_order_workspace(void) { return 256 + 2 * 1024 * sizeof(unsigned); }

int chem_cost_order(chem_mech_t m, int64_t n_cells, const int32_t* cost, int32_t* order, void* ws, size_t ws_bytes,
                    void* stream) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (n_cells < 0 || n_cells > INT32_MAX) return fail(CHEM_EARG, "n_cells out of range");
  if (n_cells == 0) return 0;
  if (!cost || !order) return fail(CHEM_EARG, "NULL array");
  if (!ws || ws_bytes < chem_cost_order_workspace() || (((uintptr_t)ws) & 255))
    return fail(CHEM_EWS, "cost-order workspace of %zu aligned bytes needed", chem_cost_order_workspace());
  if (int rc = make_current(m)) return rc;
  Module* mod;
  if (int rc = resolve(m, nullptr, &mod)) return rc;
  CUstream s = (CUstream)stream;
  unsigned* bins = (unsigned*)ws;
  unsigned* starts = bins + 1024;
  CU_TRY(drv::cuMemsetD32Async((CUdeviceptr)bins, 0, 1024, s));
  long long nc = n_cells;
  const unsigned grid = (unsigned)((n_cells + 255) / 256);
  void* ha[] = {&nc, (void*)&cost, &bins};
  CU_TRY(drv::cuLaunchKernel(mod->f_ohist, grid, 1, 1, 256, 1, 1, 0, s, ha, nullptr));
  void* sa[] = {&bins, &starts};
  CU_TRY(drv::cuLaunchKernel(mod->f_oscan, 1, 1, 1, 1024, 1, 1, 0, s, sa, nullptr));
  void* ca[] = {&nc, (void*)&cost, &starts, &order};
  CU_TRY(drv::cuLaunchKernel(mod->f_oscat, grid, 1, 1, 256, 1, 1, 0, s, ca, nullptr));
  return 0;
}

// Throughput probe of the FP64 pipe: independent FMA chains (8 per thread), and chains of exp and
// log (4 per thread), over a grid of 4 blocks x 256 threads per SM.  Costs are reported per call
// in units of one FMA's pipe time.
static const char* const kFp64ProbeSource = R"PROBE(
extern "C" __global__ void __launch_bounds__(256) probe_fma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1e-3 * threadIdx.x + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
extern "C" __global__ void __launch_bounds__(256) probe_exp(double* out, int iters) {
  double x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) x[k] = 1e-4 * threadIdx.x + 0.1 * k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = exp(-x[k]);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}
extern "C" __global__ void __launch_bounds__(256) probe_log(double* out, int iters) {
  double x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) x[k] = 1e-4 * threadIdx.x + 0.1 * k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = log(x[k] + 2.5);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}
)PROBE";

int chem_fp64_probe(void* stream, double* dfma_tflops, double* exp_cost, double* log_cost) {
  if (!drv::load()) return fail(CHEM_ECUDA, "%s", drv::load_error.c_str());
  CU_TRY(drv::cuInit(0));
  CUcontext ctx = nullptr;
  CU_TRY(drv::cuCtxGetCurrent(&ctx));
  if (!ctx) {
    CUdevice dev;
    CU_TRY(drv::cuDeviceGet(&dev, 0));
    CU_TRY(drv::cuDevicePrimaryCtxRetain(&ctx, dev));
    CU_TRY(drv::cuCtxSetCurrent(ctx));
  }
  CUdevice dev;
  CU_TRY(drv::cuCtxGetDevice(&dev));
  int n_sm = 0;
  CU_TRY(drv::cuDeviceGetAttribute(&n_sm, CU_DEVICE_ATTRIBUTE_MULTIPROCESSOR_COUNT, dev));
  std::string cubin, log;
  if (int rc = nvrtc_compile(kFp64ProbeSource, "chem_fp64_probe.cu", &cubin, &log)) return rc;
  CUmodule mod;
  CU_TRY(drv::cuModuleLoadData(&mod, cubin.data()));
  struct Unload { CUmodule m; ~Unload() { drv::cuModuleUnload(m); } } unload{mod};
  CUfunction f_fma, f_exp, f_log;
  CU_TRY(drv::cuModuleGetFunction(&f_fma, mod, "probe_fma"));
  CU_TRY(drv::cuModuleGetFunction(&f_exp, mod, "probe_exp"));
  CU_TRY(drv::cuModuleGetFunction(&f_log, mod, "probe_log"));
  const unsigned grid = (unsigned)n_sm * 4, tpb = 256;
  CUdeviceptr out = 0;
  CU_TRY(drv::cuMemAlloc(&out, sizeof(double) * grid * tpb));
  struct Free { CUdeviceptr p; ~Free() { if (p) drv::cuMemFree(p); } } guard{out};
  CUstream s = (CUstream)stream;
  CUevent e0, e1;
  CU_TRY(drv::cuEventCreate(&e0, 0));
  CU_TRY(drv::cuEventCreate(&e1, 0));
  // best of 3 timed launches after one warm-up, seconds
  auto timed = [&](CUfunction f, void** args, double* sec) -> int {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      CU_TRY(drv::cuEventRecord(e0, s));
      CU_TRY(drv::cuLaunchKernel(f, grid, 1, 1, tpb, 1, 1, 0, s, args, nullptr));
      CU_TRY(drv::cuEventRecord(e1, s));
      CU_TRY(drv::cuEventSynchronize(e1));
      float ms = 0;
      CU_TRY(drv::cuEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < best) best = ms;
    }
    *sec = best * 1e-3;
    return 0;
  };
  int it_fma = 8192, it_tr = 1024;
  double a = 0.999999, b = 1e-6;
  double t_fma = 0, t_exp = 0, t_log = 0;
  void* af[] = {&out, &it_fma, &a, &b};
  void* ae[] = {&out, &it_tr};
  int rc = timed(f_fma, af, &t_fma);
  if (!rc) rc = timed(f_exp, ae, &t_exp);
  if (!rc) rc = timed(f_log, ae, &t_log);
  drv::cuEventDestroy(e0);
  drv::cuEventDestroy(e1);
  if (rc) return rc;
  const double threads = (double)grid * tpb;
  const double n_fma = threads * 8.0 * it_fma, n_tr = threads * 4.0 * it_tr;
  const double per_fma = t_fma / n_fma;
  if (dfma_tflops) *dfma_tflops = 2.0 * n_fma / t_fma * 1e-12;
  if (exp_cost) *exp_cost = (t_exp / n_tr) / per_fma;
  if (log_cost) *log_cost = (t_log / n_tr) / per_fma;  // includes the argument's add (one FP64 op)
  return 0;
}

int chem_autotune(chem_mech_t m, int64_t n_cells, const double* T, const double* P, const double* Y, int64_t ld,
                  double dt, double rtol, double atol, void* stream, int32_t* team_out, int32_t* block_out,
                  float* ms_out) {
  if (!m) return fail(CHEM_EARG, "NULL mechanism");
  if (int rc = check_cells(n_cells, ld)) return rc;
  if (n_cells == 0 || !T || !P || !Y) return fail(CHEM_EARG, "autotune needs a non-empty sample");
  if (int rc = make_current(m)) return rc;
  const int ns = (int)m->data.sp.size();
  CUstream s = (CUstream)stream;
  std::vector<std::pair<int, int>> cand = {{32, 32}, {32, 64}, {64, 64}, {128, 128}, {256, 256}};
  // several cells per warp for small mechanisms
  if (ns <= 32) cand.insert(cand.begin(), {{4, 64}, {8, 64}, {8, 128}, {16, 128}});
  if (ns <= 64) cand.insert(cand.begin(), {16, 64});
  if (ns <= 16) cand.insert(cand.begin(), {1, 32});
  // compile the candidates not loaded yet in parallel host threads (NVRTC is thread-safe); the
  // modules are then loaded one by one
  std::vector<std::string> cubins(cand.size());
  {
    int max_optin = 0;
    CUdevice dev;
    CU_TRY(drv::cuCtxGetDevice(&dev));
    CU_TRY(drv::cuDeviceGetAttribute(&max_optin, CU_DEVICE_ATTRIBUTE_MAX_SHARED_MEMORY_PER_BLOCK_OPTIN, dev));
    std::vector<int> todo;
    {
      std::lock_guard<std::mutex> lk(m->mu);
      for (size_t i = 0; i < cand.size(); ++i)
        if (!m->modules.count(std::make_tuple(cand[i].first, cand[i].second, 0)) &&
            check_config(cand[i].first, cand[i].second) == 0 &&
            smem_bytes(m->data, cand[i].first, cand[i].second, 0) <= max_optin)
          todo.push_back((int)i);
    }
    std::vector<std::thread> th;
    for (int i : todo)
      th.emplace_back([&, i] {
        std::string lg;
        if (build_cubin(m->data, cand[i].first, cand[i].second, false, 0, m->cache_dir.c_str(), false,
                        &cubins[i], &lg))
          cubins[i].clear();
      });
    for (auto& t : th) t.join();
  }
  // the sample: enough cells for four waves of the widest candidate's resident teams (at least
  // 4096), so that every candidate is timed at full occupancy
  std::vector<Module*> mods(cand.size(), nullptr);
  int64_t resident = 0;
  for (size_t ci = 0; ci < cand.size(); ++ci) {
    if (get_module(m, cand[ci].first, cand[ci].second, &mods[ci], false, 0, &cubins[ci]) != 0) {
      mods[ci] = nullptr;  // does not fit: skip
      continue;
    }
    resident = std::max<int64_t>(resident, (int64_t)m->n_sm * mods[ci]->occ * teams_per_block(mods[ci]));
  }
  const int64_t n = std::min<int64_t>(n_cells, std::max<int64_t>(4096, 4 * resident));
  // private copy of the sample: T, P, Y [ns][n], h, workspace
  const size_t oT = 0, oP = align256(8 * n), oY = align256(oP + 8 * n), oY0 = align256(oY + 8 * n * ns),
               oT0 = align256(oY0 + 8 * n * ns), oW = align256(oT0 + 8 * n), total = oW + 256;
  CUdeviceptr buf = 0;
  CU_TRY(drv::cuMemAlloc(&buf, total));
  struct Free { CUdeviceptr p; ~Free() { if (p) drv::cuMemFree(p); } } guard{buf};
  CU_TRY(drv::cuMemcpyDtoDAsync(buf + oT0, (CUdeviceptr)T, 8 * n, s));
  CU_TRY(drv::cuMemcpyDtoDAsync(buf + oP, (CUdeviceptr)P, 8 * n, s));
  for (int k = 0; k < ns; ++k)
    CU_TRY(drv::cuMemcpyDtoDAsync(buf + oY0 + 8 * n * k, (CUdeviceptr)(Y + (size_t)k * ld), 8 * n, s));
  CUevent e0, e1;
  CU_TRY(drv::cuEventCreate(&e0, 0));
  CU_TRY(drv::cuEventCreate(&e1, 0));
  float best = 1e30f;
  int bt = m->default_team, bb = m->default_tpb;
  for (size_t ci = 0; ci < cand.size(); ++ci) {
    const auto& c = cand[ci];
    if (!mods[ci]) continue;
    chem_int_opts o{};
    o.team = c.first;
    o.block = c.second;
    float ms = 0;
    for (int rep = 0; rep < 2; ++rep) {
      CU_TRY(drv::cuMemcpyDtoDAsync(buf + oT, buf + oT0, 8 * n, s));
      CU_TRY(drv::cuMemcpyDtoDAsync(buf + oY, buf + oY0, 8 * n * ns, s));
      CU_TRY(drv::cuEventRecord(e0, s));
      int rc = chem_integrate(m, n, (double*)(buf + oT), (const double*)(buf + oP), (double*)(buf + oY), n, dt, rtol,
                              atol, nullptr, nullptr, &o, (void*)(buf + oW), 256, stream);
      if (rc) return rc;
      CU_TRY(drv::cuEventRecord(e1, s));
      CU_TRY(drv::cuEventSynchronize(e1));
      CU_TRY(drv::cuEventElapsedTime(&ms, e0, e1));
    }
    if (ms < best) { best = ms; bt = c.first; bb = c.second; }
  }
  drv::cuEventDestroy(e0);
  drv::cuEventDestroy(e1);
  m->default_team = bt;
  m->default_tpb = bb;
  if (team_out) *team_out = bt;
  if (block_out) *block_out = bb;
  if (ms_out) *ms_out = best;
  return 0;
}

}  // extern "C"
