// CPU oracle for the batched ROS4 chemistry integrator.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
// reference leg load this library.  The CUDA path shares no code with it: it has its own spec
// parser, thermodynamics, rates, Jacobian, LU and integrator.
//
// Plain, slow, FP64 C++.  Every routine is templated on the scalar type so that the same code
// runs on double, on std::complex<double> (complex-step derivatives) and on forward-mode dual
// numbers.  Nothing is blocked, fused or reordered beyond the definitions it follows.
//
// What it computes (Curtis, Niemeyer & Sung, "Accelerating reactive-flow simulations using
// vectorized chemistry integration"):
//   * state y = [T, n_1 .. n_{Ns-1}] with the bath gas (last species) closed implicitly,
//     Sec. 2.1, Eq. (e:state_vec) and Eq. (e:n_nsp).  Reading: unit-mass basis, so the closure
//     is mass conservation n_Ns = (1 - sum_k W_k n_k) / W_Ns and V = n_tot R T / P, which is
//     the same closure as Eq. (e:n_nsp) for a mass-balanced mechanism.
//   * source terms dy/dt = f(y), Eq. (e:dphidt); species rates from mass action with
//     Arrhenius, third-body, Lindemann and Troe falloff rate constants; reverse rates from
//     NASA-7 equilibrium constants (the paper delegates these textbook forms to pyJac, Sec. 2.1).
//   * the Jacobian J_ij = d f_i / d y_j, Eq. (e:jac), formed here by forward-mode dual numbers
//     through f (the exact derivative of the definition).
//   * the s-stage Rosenbrock method in its transformed form, Sec. 2.3, Eq. (e:ros) and the
//     transformation below it, with the Hairer-Wanner L-stable ROS4 coefficients, embedded
//     error estimate and adaptive step size.
//
// Parity pins for every function live in tests/test_oracle_*.py.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

namespace orc {

constexpr double R_U = 8314.462618;          // J/(kmol K)
constexpr double R_CAL = 1.987204258640832;   // cal/(mol K)
constexpr double P_ATM = 101325.0;            // Pa
constexpr double CGS_TO_SI = 1e-3;            // 1 cm^3/mol = 1e-3 m^3/kmol

enum Kind { ELEM = 0, THIRD = 1, LIND = 2, TROE = 3 };

struct Species {
  std::string name;
  double W = 0;
  std::vector<int> counts;
  double Tlow = 0, Tmid = 0, Thigh = 0, hf_R = 0, s_R = 0;
  double lo[7] = {0}, hi[7] = {0};
};

struct Reaction {
  int kind = ELEM;
  std::vector<int> rsp, rnu, psp, pnu;
  double lnA = 0, b = 0, theta = 0;   // SI units, theta = Ea / R [K]
  std::vector<double> eff;            // third-body efficiencies, one per species
  double lnA0 = 0, b0 = 0, theta0 = 0;
  double troe_a = 0, troe_T3 = 0, troe_T1 = 0, troe_T2 = 0;
};

struct Mech {
  std::vector<std::string> elements;
  std::vector<Species> sp;
  std::vector<Reaction> rx;
  int ns = 0, nr = 0;
};

// ------------------------------------------------------------------------------ spec parser

static Mech parse(const std::string& path) {
  std::ifstream in(path);
  if (!in) throw std::runtime_error("cannot open " + path);
  Mech m;
  std::map<std::string, int> index;
  std::string line;
  Species* cur_sp = nullptr;
  Reaction* cur_rx = nullptr;
  int declared_sp = -1, declared_rx = -1;
  auto species_of = [&](const std::string& name) {
    auto it = index.find(name);
    if (it == index.end()) throw std::runtime_error("unknown species " + name);
    return it->second;
  };
  while (std::getline(in, line)) {
    auto hash = line.find('#');
    if (hash != std::string::npos) line = line.substr(0, hash);
    std::istringstream ss(line);
    std::string tag;
    if (!(ss >> tag)) continue;
    if (tag == "MECHANISM") {
    } else if (tag == "ELEMENTS") {
      std::string e;
      while (ss >> e) m.elements.push_back(e);
    } else if (tag == "SPECIES") {
      ss >> declared_sp;
    } else if (tag == "SP") {
      Species s;
      ss >> s.name >> s.W;
      s.counts.resize(m.elements.size());
      for (auto& c : s.counts) ss >> c;
      ss >> s.Tlow >> s.Tmid >> s.Thigh >> s.hf_R >> s.s_R;
      if (!ss) throw std::runtime_error("bad SP line: " + line);
      index[s.name] = (int)m.sp.size();
      m.sp.push_back(s);
      cur_sp = &m.sp.back();
    } else if (tag == "LO" || tag == "HI") {
      if (!cur_sp) throw std::runtime_error("LO/HI before SP");
      double* a = tag == "LO" ? cur_sp->lo : cur_sp->hi;
      for (int i = 0; i < 7; ++i) ss >> a[i];
      if (!ss) throw std::runtime_error("bad NASA line: " + line);
    } else if (tag == "REACTIONS") {
      ss >> declared_rx;
      m.ns = (int)m.sp.size();
      m.rx.reserve(declared_rx > 0 ? declared_rx : 0);
    } else if (tag == "R") {
      Reaction r;
      std::string kind;
      ss >> kind;
      if (kind == "ELEM") r.kind = ELEM;
      else if (kind == "THIRD") r.kind = THIRD;
      else if (kind == "LIND") r.kind = LIND;
      else if (kind == "TROE") r.kind = TROE;
      else throw std::runtime_error("unknown reaction type " + kind);
      int n;
      std::string name;
      int nu;
      ss >> n;
      for (int i = 0; i < n; ++i) { ss >> name >> nu; r.rsp.push_back(species_of(name)); r.rnu.push_back(nu); }
      ss >> n;
      for (int i = 0; i < n; ++i) { ss >> name >> nu; r.psp.push_back(species_of(name)); r.pnu.push_back(nu); }
      double A, b, Ea;
      ss >> A >> b >> Ea;
      if (!ss) throw std::runtime_error("bad R line: " + line);
      int order = 0;
      for (int v : r.rnu) order += v;
      if (r.kind == THIRD) order += 1;
      // Chemkin units (cm^3/mol)^(order-1)/s to SI (m^3/kmol)^(order-1)/s
      r.lnA = std::log(A) + (order - 1) * std::log(CGS_TO_SI);
      r.b = b;
      r.theta = Ea / R_CAL;
      r.eff.assign(m.sp.size(), 1.0);
      m.rx.push_back(r);
      cur_rx = &m.rx.back();
    } else if (tag == "EFF") {
      if (!cur_rx) throw std::runtime_error("EFF before R");
      int n;
      ss >> n;
      for (int i = 0; i < n; ++i) {
        std::string name;
        double e;
        ss >> name >> e;
        cur_rx->eff[species_of(name)] = e;
      }
    } else if (tag == "LOW") {
      if (!cur_rx) throw std::runtime_error("LOW before R");
      double A0, b0, Ea0;
      ss >> A0 >> b0 >> Ea0;
      int order = 1;  // low-pressure limit carries the +M
      for (int v : cur_rx->rnu) order += v;
      cur_rx->lnA0 = std::log(A0) + (order - 1) * std::log(CGS_TO_SI);
      cur_rx->b0 = b0;
      cur_rx->theta0 = Ea0 / R_CAL;
    } else if (tag == "TROE") {
      if (!cur_rx) throw std::runtime_error("TROE before R");
      ss >> cur_rx->troe_a >> cur_rx->troe_T3 >> cur_rx->troe_T1 >> cur_rx->troe_T2;
    } else if (tag == "END") {
      break;
    } else {
      throw std::runtime_error("unknown record " + tag);
    }
  }
  m.ns = (int)m.sp.size();
  m.nr = (int)m.rx.size();
  if (declared_sp != m.ns || declared_rx != m.nr) throw std::runtime_error("count mismatch in spec");
  return m;
}

// ------------------------------------------------------------------------------ scalar types

inline double re(double x) { return x; }
inline double re(const std::complex<double>& x) { return x.real(); }

// forward-mode dual number with M tangent directions
template <class S, int M>
struct Dual {
  S v;
  S d[M];
  Dual() : v(0.0) { for (int i = 0; i < M; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < M; ++i) d[i] = 0.0; }
  Dual(const S& x, int) : v(x) { for (int i = 0; i < M; ++i) d[i] = 0.0; }
};
template <class S, int M> double re(const Dual<S, M>& x) { return re(x.v); }

template <class S, int M> Dual<S, M> operator+(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v + b.v; for (int i = 0; i < M; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <class S, int M> Dual<S, M> operator-(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v - b.v; for (int i = 0; i < M; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <class S, int M> Dual<S, M> operator-(const Dual<S, M>& a) {
  Dual<S, M> r; r.v = -a.v; for (int i = 0; i < M; ++i) r.d[i] = -a.d[i]; return r; }
template <class S, int M> Dual<S, M> operator*(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v * b.v; for (int i = 0; i < M; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <class S, int M> Dual<S, M> operator/(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v / b.v;
  for (int i = 0; i < M; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <class S, int M> Dual<S, M> operator+(const Dual<S, M>& a, double b) { Dual<S, M> r = a; r.v = r.v + b; return r; }
template <class S, int M> Dual<S, M> operator+(double b, const Dual<S, M>& a) { return a + b; }
template <class S, int M> Dual<S, M> operator-(const Dual<S, M>& a, double b) { Dual<S, M> r = a; r.v = r.v - b; return r; }
template <class S, int M> Dual<S, M> operator-(double b, const Dual<S, M>& a) { return (-a) + b; }
template <class S, int M> Dual<S, M> operator*(const Dual<S, M>& a, double b) {
  Dual<S, M> r; r.v = a.v * b; for (int i = 0; i < M; ++i) r.d[i] = a.d[i] * b; return r; }
template <class S, int M> Dual<S, M> operator*(double b, const Dual<S, M>& a) { return a * b; }
template <class S, int M> Dual<S, M> operator/(const Dual<S, M>& a, double b) {
  Dual<S, M> r; r.v = a.v / b; for (int i = 0; i < M; ++i) r.d[i] = a.d[i] / b; return r; }
template <class S, int M> Dual<S, M> operator/(double b, const Dual<S, M>& a) { return Dual<S, M>(b) / a; }
template <class S, int M> Dual<S, M> exp(const Dual<S, M>& a) {
  using std::exp;
  Dual<S, M> r; r.v = exp(a.v); for (int i = 0; i < M; ++i) r.d[i] = r.v * a.d[i]; return r; }
template <class S, int M> Dual<S, M> log(const Dual<S, M>& a) {
  using std::log;
  Dual<S, M> r; r.v = log(a.v); for (int i = 0; i < M; ++i) r.d[i] = a.d[i] / a.v; return r; }
template <class S, int M> Dual<S, M> log10(const Dual<S, M>& a) { return log(a) / std::log(10.0); }

template <class S> S pow_int(const S& x, int k) {
  S r = 1.0;
  for (int i = 0; i < k; ++i) r = r * x;
  return r;
}

// ------------------------------------------------------------------------------ thermo
// NASA-7: cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4,
//         h/(RT) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T,
//         s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7.
// Low range for T < Tmid, high range otherwise.

template <class S>
void thermo(const Species& s, const S& T, S& cp, S& hRT, S& sR) {
  using std::log;
  const double* a = re(T) < s.Tmid ? s.lo : s.hi;
  S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
  cp = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
  hRT = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
  sR = a[0] * log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
}

// ------------------------------------------------------------------------------ rates and f

template <class S>
struct Rates {
  std::vector<S> C, kf, kr, qf, qr, omega;  // qf/qr include the [M] factor of THIRD reactions
  S V, T;
};

// Species concentrations, rate constants, rates of progress and net production rates
// omega_k [kmol/m^3/s] of one cell at state y (size Ns) and pressure P.
template <class S>
void rates(const Mech& m, const S* y, double P, const S* lnA, Rates<S>& out) {
  using std::exp;
  using std::log;
  using std::log10;
  const int ns = m.ns;
  const S T = y[0];
  std::vector<S> n(ns);
  S mass = 0.0;
  for (int k = 0; k < ns - 1; ++k) { n[k] = y[1 + k]; mass = mass + m.sp[k].W * n[k]; }
  n[ns - 1] = (1.0 - mass) / m.sp[ns - 1].W;  // bath gas from mass conservation
  S ntot = 0.0;
  for (int k = 0; k < ns; ++k) ntot = ntot + n[k];
  const S V = ntot * R_U * T / P;  // m^3 per kg of mixture
  out.V = V;
  out.T = T;
  out.C.assign(ns, S(0.0));
  for (int k = 0; k < ns; ++k) out.C[k] = n[k] / V;
  std::vector<S> cp(ns), hRT(ns), sR(ns);
  for (int k = 0; k < ns; ++k) thermo(m.sp[k], T, cp[k], hRT[k], sR[k]);
  out.kf.assign(m.nr, S(0.0));
  out.kr.assign(m.nr, S(0.0));
  out.qf.assign(m.nr, S(0.0));
  out.qr.assign(m.nr, S(0.0));
  out.omega.assign(ns, S(0.0));
  const S lnT = log(T);
  for (int r = 0; r < m.nr; ++r) {
    const Reaction& R = m.rx[r];
    const S lnAr = lnA ? lnA[r] : S(R.lnA);
    S kf = exp(lnAr + R.b * lnT - R.theta / T);
    S Mconc = 0.0;
    if (R.kind != ELEM)
      for (int k = 0; k < ns; ++k) Mconc = Mconc + R.eff[k] * out.C[k];
    if (R.kind == LIND || R.kind == TROE) {
      const S k0 = exp(R.lnA0 + R.b0 * lnT - R.theta0 / T);
      S Pr = k0 * Mconc / kf;
      if (re(Pr) < 1e-300) Pr = S(1e-300);
      S F = 1.0;
      if (R.kind == TROE) {
        S Fcent = (1.0 - R.troe_a) * exp(-T / R.troe_T3) + R.troe_a * exp(-T / R.troe_T1);
        if (R.troe_T2 > 0) Fcent = Fcent + exp(-R.troe_T2 / T);
        const S lFc = log10(Fcent);
        const S c = -0.4 - 0.67 * lFc;
        const S nn = 0.75 - 1.27 * lFc;
        const S x = log10(Pr) + c;
        const S f1 = x / (nn - 0.14 * x);
        const S lF = lFc / (1.0 + f1 * f1);
        F = exp(lF * std::log(10.0));
      }
      kf = kf * (Pr / (1.0 + Pr)) * F;
    }
    // equilibrium constant in concentration units from the standard Gibbs energy change
    S dG = 0.0;  // sum nu (s/R - h/RT)
    int dnu = 0;
    for (size_t i = 0; i < R.psp.size(); ++i) { dG = dG + double(R.pnu[i]) * (sR[R.psp[i]] - hRT[R.psp[i]]); dnu += R.pnu[i]; }
    for (size_t i = 0; i < R.rsp.size(); ++i) { dG = dG - double(R.rnu[i]) * (sR[R.rsp[i]] - hRT[R.rsp[i]]); dnu -= R.rnu[i]; }
    S Kc = exp(dG) * exp(double(dnu) * log(P_ATM / (R_U * T)));
    S kr = kf / Kc;
    S qf = kf, qr = kr;
    for (size_t i = 0; i < R.rsp.size(); ++i) qf = qf * pow_int(out.C[R.rsp[i]], R.rnu[i]);
    for (size_t i = 0; i < R.psp.size(); ++i) qr = qr * pow_int(out.C[R.psp[i]], R.pnu[i]);
    if (R.kind == THIRD) { qf = qf * Mconc; qr = qr * Mconc; }
    out.kf[r] = kf;
    out.kr[r] = kr;
    out.qf[r] = qf;
    out.qr[r] = qr;
    const S q = qf - qr;
    for (size_t i = 0; i < R.rsp.size(); ++i) out.omega[R.rsp[i]] = out.omega[R.rsp[i]] - double(R.rnu[i]) * q;
    for (size_t i = 0; i < R.psp.size(); ++i) out.omega[R.psp[i]] = out.omega[R.psp[i]] + double(R.pnu[i]) * q;
  }
  (void)n;
}

// f(y): dT/dt from the adiabatic constant-pressure energy balance, dn_k/dt = V omega_k.
template <class S>
void source(const Mech& m, const S* y, double P, const S* lnA, S* f) {
  Rates<S> R;
  rates(m, y, P, lnA, R);
  const int ns = m.ns;
  const S T = y[0];
  std::vector<S> cp(ns), hRT(ns), sR(ns);
  for (int k = 0; k < ns; ++k) thermo(m.sp[k], T, cp[k], hRT[k], sR[k]);
  S mass = 0.0;
  for (int k = 0; k < ns - 1; ++k) mass = mass + m.sp[k].W * y[1 + k];
  S heat = 0.0, cpmix = 0.0;  // sum_k h_k dn_k/dt / R and sum_k n_k cp_k / R
  for (int k = 0; k < ns; ++k) {
    const S nk = k < ns - 1 ? y[1 + k] : (1.0 - mass) / m.sp[ns - 1].W;
    heat = heat + hRT[k] * T * R.V * R.omega[k];
    cpmix = cpmix + nk * cp[k];
  }
  f[0] = -heat / cpmix;
  for (int k = 0; k < ns - 1; ++k) f[1 + k] = R.V * R.omega[k];
}

// J = df/dy by forward-mode dual numbers: the j-th tangent direction is e_j.
template <int M, class S>
void jacobian_dual(const Mech& m, const S* y, double P, const S* lnA, S* J) {
  typedef Dual<S, M> D;
  const int N = m.ns;
  std::vector<D> yd(N), fd(N), lnAd;
  for (int j = 0; j < N; ++j) { yd[j] = D(y[j], 0); yd[j].d[j] = 1.0; }
  if (lnA) { lnAd.resize(m.nr); for (int r = 0; r < m.nr; ++r) lnAd[r] = D(lnA[r], 0); }
  source(m, yd.data(), P, lnA ? lnAd.data() : (const D*)nullptr, fd.data());
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) J[i * N + j] = fd[i].d[j];
}

template <class S>
void jacobian(const Mech& m, const S* y, double P, const S* lnA, S* J) {
  if (m.ns <= 16) jacobian_dual<16>(m, y, P, lnA, J);
  else if (m.ns <= 64) jacobian_dual<64>(m, y, P, lnA, J);
  else if (m.ns <= 128) jacobian_dual<128>(m, y, P, lnA, J);
  else throw std::runtime_error("oracle Jacobian supports at most 128 species");
}

// ------------------------------------------------------------------------------ linear algebra
// LU with partial pivoting (largest |real part|, lowest row on ties); row-major n x n, in place.

template <class S>
void lu_factor(int n, S* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(re(A[k * n + k]));
    for (int i = k + 1; i < n; ++i) {
      const double v = std::fabs(re(A[i * n + k]));
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      A[i * n + k] = A[i * n + k] / A[k * n + k];
      for (int j = k + 1; j < n; ++j) A[i * n + j] = A[i * n + j] - A[i * n + k] * A[k * n + j];
    }
  }
}

template <class S>
void lu_solve(int n, const S* LU, const int* piv, S* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] = b[i] - LU[i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] = b[i] - LU[i * n + j] * b[j];
    b[i] = b[i] / LU[i * n + i];
  }
}

// ------------------------------------------------------------------------------ ROS4
// Hairer & Wanner, Solving ODEs II, Sec. IV.7: L-stable 4-stage order-4(3) Rosenbrock method,
// written in the transformed variables of Sec. 2.3 of the paper:
//   (I/(h gamma) - J) u_i = f(y + sum_{j<i} a_ij u_j) + sum_{j<i} (c_ij / h) u_j,
//   y_new = y + sum_j m_j u_j,    error estimate = sum_j e_j u_j.
// (The paper prints sum_{j<=i} and c = gamma I - Gamma^-1; the diagonal belongs to the left-hand
//  side, so the sums run over j < i and C = diag(1/gamma) - Gamma^-1.)
struct Tableau {
  int s = 4;       // stages
  int order = 4;   // order of the main solution (the controller uses err^(-1/order))
  double gamma;
  double a[6][6];
  double c[6][6];
  double m[6];
  double e[6];
  bool erk = false;  // explicit Runge-Kutta: u_i = h f(y + sum_j a_ij u_j), no Jacobian, no c, gamma
};

static Tableau ros4_hw() {
  Tableau t{};
  t.s = 4;
  t.order = 4;
  t.gamma = 0.57282;
  t.a[1][0] = 2.0;
  t.a[2][0] = 1.867943637803922;
  t.a[2][1] = 0.2344449711399156;
  t.a[3][0] = 1.867943637803922;
  t.a[3][1] = 0.2344449711399156;
  t.c[1][0] = -7.137615036412310;
  t.c[2][0] = 2.580708087951457;
  t.c[2][1] = 0.6515950076447975;
  t.c[3][0] = -2.137148994382534;
  t.c[3][1] = -0.3214669691237626;
  t.c[3][2] = -0.6949742501781779;
  t.m[0] = 2.255570073418735;
  t.m[1] = 0.2870493262186792;
  t.m[2] = 0.4353179431840180;
  t.m[3] = 1.093502252409163;
  t.e[0] = -0.2815431932141155;
  t.e[1] = -0.07276199124938920;
  t.e[2] = -0.1082196201495311;
  t.e[3] = -1.093502252409163;
  return t;
}

// Sandu, Verwer, Blom, Spee, Carmichael & Potra (1997), "Benchmarking stiff ODE solvers for
// atmospheric chemistry problems II: Rosenbrock solvers": ROS3, 3 stages, order 3(2), L-stable.
static Tableau ros3_sandu() {
  Tableau t{};
  t.s = 3;
  t.order = 3;
  t.gamma = 0.43586652150845899941601945119356;
  t.a[1][0] = 1.0;
  t.a[2][0] = 1.0;
  t.c[1][0] = -1.0156171083877702091975600115545;
  t.c[2][0] = 4.0759956452537699824805835358067;
  t.c[2][1] = 9.2076794298330791242156818474003;
  t.m[0] = 1.0;
  t.m[1] = 6.1697947043828245592553615689730;
  t.m[2] = -0.42772256543218573326238373806514;
  t.e[0] = 0.5;
  t.e[1] = -2.9079558716805469821718236208017;
  t.e[2] = 0.22354069897811569627360909276199;
  return t;
}

// Sandu et al. (1997): RODAS3, 4 stages, order 3(2), stiffly accurate.
static Tableau rodas3_sandu() {
  Tableau t{};
  t.s = 4;
  t.order = 3;
  t.gamma = 0.5;
  t.a[2][0] = 2.0;
  t.a[3][0] = 2.0;
  t.a[3][2] = 1.0;
  t.c[1][0] = 4.0;
  t.c[2][0] = 1.0;
  t.c[2][1] = -1.0;
  t.c[3][0] = 1.0;
  t.c[3][1] = -1.0;
  t.c[3][2] = -8.0 / 3.0;
  t.m[0] = 2.0;
  t.m[2] = 1.0;
  t.m[3] = 1.0;
  t.e[3] = 1.0;
  return t;
}

// Hairer & Wanner, Solving ODEs II, Sec. VI.4: RODAS4, 6 stages, order 4(3), stiffly accurate.
static Tableau rodas4_hw() {
  Tableau t{};
  t.s = 6;
  t.order = 4;
  t.gamma = 0.25;
  t.a[1][0] = 1.544;
  t.a[2][0] = 0.9466785280815826;
  t.a[2][1] = 0.2557011698983284;
  t.a[3][0] = 3.314825187068521;
  t.a[3][1] = 2.896124015972201;
  t.a[3][2] = 0.9986419139977817;
  t.a[4][0] = 1.221224509226641;
  t.a[4][1] = 6.019134481288629;
  t.a[4][2] = 12.53708332932087;
  t.a[4][3] = -0.6878860361058950;
  for (int j = 0; j < 4; ++j) t.a[5][j] = t.a[4][j];
  t.a[5][4] = 1.0;
  t.c[1][0] = -5.6688;
  t.c[2][0] = -2.430093356833875;
  t.c[2][1] = -0.2063599157091915;
  t.c[3][0] = -0.1073529058151375;
  t.c[3][1] = -9.594562251023355;
  t.c[3][2] = -20.47028614809616;
  t.c[4][0] = 7.496443313967647;
  t.c[4][1] = -10.24680431464352;
  t.c[4][2] = -33.99990352819905;
  t.c[4][3] = 11.70890893206160;
  t.c[5][0] = 8.083246795921522;
  t.c[5][1] = -7.981132988064893;
  t.c[5][2] = -31.52159432874371;
  t.c[5][3] = 16.31930543123136;
  t.c[5][4] = -6.058818238834054;
  for (int j = 0; j < 4; ++j) t.m[j] = t.a[4][j];
  t.m[4] = 1.0;
  t.m[5] = 1.0;
  t.e[5] = 1.0;
  return t;
}

// Rosenbrock methods of Table T:solvers by id: 0 ROS4 (default), 1 ROS3, 2 RODAS3, 3 RODAS4
// Runge-Kutta-Fehlberg 4(5) (Fehlberg 1969; Hairer, Norsett and Wanner, Solving ODEs I, Table
// II.5.1), the explicit solver of the paper's Table T:solvers.  Written in the increment form
// u_i = h k_i so that it shares y_new = y + sum m_j u_j and the error sum e_j u_j with the
// Rosenbrock methods.  Reading (the paper does not say which solution is propagated): the
// fifth-order solution is carried (local extrapolation), the difference to the embedded
// fourth-order solution is the error estimate, so the controller exponent is 1/5.
static Tableau rkf45_fehlberg() {
  Tableau t{};
  t.s = 6;
  t.order = 5;
  t.erk = true;
  t.gamma = 0.0;
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

// ROS2 of Verwer, Spee, Blom & Hundsdorfer (1999), "A second-order Rosenbrock method applied to
// photochemical dispersion problems": (I - g h W) k1 = f(y), (I - g h W) k2 = f(y + h k1) - 2 k1,
// y1 = y + 3/2 h k1 + 1/2 h k2, g = 1 + 1/sqrt(2).  Second order for ANY matrix W (a W-method,
// the class the paper names for reusing Jacobians and their factorisations), L-stable for this
// g.  Error estimate: the difference to the first-order y + h k1, i.e. h/2 (k1 + k2).  In the
// transformed variables u_i = g h k_i of the other methods: a21 = 1/g, c21 = -2/g,
// m = (3/(2g), 1/(2g)), e = (1/(2g), 1/(2g)).
static Tableau ros2_w() {
  Tableau t{};
  t.s = 2;
  t.order = 2;
  t.gamma = 1.0 + 1.0 / std::sqrt(2.0);
  const double g = t.gamma;
  t.a[1][0] = 1.0 / g;
  t.c[1][0] = -2.0 / g;
  t.m[0] = 1.5 / g;
  t.m[1] = 0.5 / g;
  t.e[0] = 0.5 / g;
  t.e[1] = 0.5 / g;
  return t;
}

static Tableau tableau_by_id(int id) {
  switch (id) {
    case 1: return ros3_sandu();
    case 2: return rodas3_sandu();
    case 3: return rodas4_hw();
    case 4: return rkf45_fehlberg();
    case 5: return ros2_w();
    default: return ros4_hw();
  }
}

// An ODE system y' = F(y) with Jacobian; Sys provides rhs() and jac() for scalar S.
template <class S>
struct ChemSys {
  const Mech& m;
  double P;
  const S* lnA;
  int n() const { return m.ns; }
  void rhs(const S* y, S* f) const { source(m, y, P, lnA, f); }
  void jac(const S* y, S* J) const { jacobian(m, y, P, lnA, J); }
};

template <class S>
struct LinSys {  // y' = A y
  int N;
  const double* A;
  int n() const { return N; }
  void rhs(const S* y, S* f) const {
    for (int i = 0; i < N; ++i) { f[i] = 0.0; for (int j = 0; j < N; ++j) f[i] = f[i] + A[i * N + j] * y[j]; }
  }
  void jac(const S*, S* J) const { for (int i = 0; i < N * N; ++i) J[i] = A[i]; }
};

// One explicit Runge-Kutta step (tb.erk): u_i = h f(y + sum_{j<i} a_ij u_j).
template <class S, class Sys>
void erk_step(const Sys& sys, const Tableau& tb, const S* y, double h, S* ynew, S* err) {
  const int N = sys.n();
  std::vector<S> u(tb.s * N), Y(N), F(N);
  for (int i = 0; i < tb.s; ++i) {
    for (int k = 0; k < N; ++k) {
      Y[k] = y[k];
      for (int j = 0; j < i; ++j) Y[k] = Y[k] + tb.a[i][j] * u[j * N + k];
    }
    sys.rhs(Y.data(), F.data());
    for (int k = 0; k < N; ++k) u[i * N + k] = h * F[k];
  }
  for (int k = 0; k < N; ++k) {
    ynew[k] = y[k];
    err[k] = 0.0;
    for (int j = 0; j < tb.s; ++j) {
      ynew[k] = ynew[k] + tb.m[j] * u[j * N + k];
      err[k] = err[k] + tb.e[j] * u[j * N + k];
    }
  }
}

// One ROS4 step of size h from y: ynew and the embedded error vector (an explicit tableau
// takes the explicit step).
// W (nullable): the matrix in place of J(y) (W-methods); NULL = the exact Jacobian at y.
template <class S, class Sys>
void ros4_step(const Sys& sys, const Tableau& tb, const S* y, double h, S* ynew, S* err,
               const double* W = nullptr) {
  if (tb.erk) {
    erk_step(sys, tb, y, h, ynew, err);
    return;
  }
  const int N = sys.n();
  std::vector<S> J(N * N), M(N * N), u(tb.s * N), Y(N), F(N);
  std::vector<int> piv(N);
  if (W)
    for (int i = 0; i < N * N; ++i) J[i] = W[i];
  else
    sys.jac(y, J.data());
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) M[i * N + j] = (i == j ? S(1.0 / (h * tb.gamma)) : S(0.0)) - J[i * N + j];
  lu_factor(N, M.data(), piv.data());
  for (int i = 0; i < tb.s; ++i) {
    for (int k = 0; k < N; ++k) {
      Y[k] = y[k];
      for (int j = 0; j < i; ++j) Y[k] = Y[k] + tb.a[i][j] * u[j * N + k];
    }
    sys.rhs(Y.data(), F.data());
    S* ui = &u[i * N];
    for (int k = 0; k < N; ++k) {
      ui[k] = F[k];
      for (int j = 0; j < i; ++j) ui[k] = ui[k] + (tb.c[i][j] / h) * u[j * N + k];
    }
    lu_solve(N, M.data(), piv.data(), ui);
  }
  for (int k = 0; k < N; ++k) {
    ynew[k] = y[k];
    err[k] = 0.0;
    for (int j = 0; j < tb.s; ++j) {
      ynew[k] = ynew[k] + tb.m[j] * u[j * N + k];
      err[k] = err[k] + tb.e[j] * u[j * N + k];
    }
  }
}

enum Status { OK = 0, MAX_STEPS = 1, H_UNDERFLOW = 2, NONFINITE = 3, SKIPPED = 4 };

struct IntOpts {
  double rtol = 1e-6, atol = 1e-10;
  int max_steps = 100000;  // attempts (accepted + rejected)
  double h_min = 1e-20;
  double T_min = 0.0;      // cells with T < T_min are left unchanged
  int fixed_steps = 0;     // > 0: that many equal steps, no error control
};

struct IntResult {
  int status = OK, attempts = 0, accepted = 0, rejected = 0;
  double h_out = 0;
};

// Weighted RMS norm of the error estimate (Hairer-Wanner scaling).
static double err_norm(int N, const double* y, const double* ynew, const double* e, double rtol, double atol) {
  double s = 0;
  for (int i = 0; i < N; ++i) {
    const double sc = atol + rtol * std::max(std::fabs(y[i]), std::fabs(ynew[i]));
    s += (e[i] / sc) * (e[i] / sc);
  }
  return std::sqrt(s / N);
}

// Integrate one system from t=0 to t=dt in place (double only).
//  * step-size factor fac = clamp(0.9 err^(-1/4), 0.2, 6), err floored at 1e-10;
//  * accept iff err <= 1; no growth on the step that follows a rejection;
//  * the step that reaches dt is cut to land on it (a step within 0.01% of the remaining
//    interval is stretched to it);
//  * h_out is the step proposal for the next call: the controller's proposal after the last
//    accepted step, or the proposal that the end-time cut shortened;
//  * fails with MAX_STEPS after max_steps attempts or H_UNDERFLOW once h < h_min.
template <class Sys>
IntResult integrate_one(const Sys& sys, const Tableau& tb, double* y, double dt, double h_in,
                        const IntOpts& o, std::vector<double>* accepted_h) {
  IntResult res;
  const int N = sys.n();
  for (int i = 0; i < N; ++i)
    if (!std::isfinite(y[i])) { res.status = NONFINITE; res.h_out = h_in; return res; }
  std::vector<double> ynew(N), e(N);
  if (o.fixed_steps > 0) {
    const double h = dt / o.fixed_steps;
    for (int s = 0; s < o.fixed_steps; ++s) {
      ros4_step(sys, tb, y, h, ynew.data(), e.data());
      for (int i = 0; i < N; ++i) y[i] = ynew[i];
      if (accepted_h) accepted_h->push_back(h);
    }
    res.attempts = res.accepted = o.fixed_steps;
    res.h_out = h;
    return res;
  }
  double t = 0.0;
  double h = h_in > 0 ? h_in : dt;
  bool reject_last = false;
  for (;;) {
    if (res.attempts >= o.max_steps) { res.status = MAX_STEPS; break; }
    if (h < o.h_min) { res.status = H_UNDERFLOW; break; }
    const bool last = t + 1.0001 * h >= dt;
    const double hh = last ? dt - t : h;
    ros4_step(sys, tb, y, hh, ynew.data(), e.data());
    res.attempts++;
    double err = err_norm(N, y, ynew.data(), e.data(), o.rtol, o.atol);
    bool finite = std::isfinite(err);
    for (int i = 0; i < N && finite; ++i) finite = std::isfinite(ynew[i]);
    double fac = finite ? std::min(6.0, std::max(0.2, 0.9 * std::pow(std::max(err, 1e-10), -1.0 / tb.order))) : 0.2;
    if (finite && err <= 1.0) {
      for (int i = 0; i < N; ++i) y[i] = ynew[i];
      res.accepted++;
      if (accepted_h) accepted_h->push_back(hh);
      if (reject_last) fac = std::min(fac, 1.0);
      reject_last = false;
      const double hnext = hh * fac;
      if (last) { h = hh < h ? h : hnext; break; }
      t += hh;
      h = hnext;
    } else {
      res.rejected++;
      reject_last = true;
      h = hh * fac;
    }
  }
  res.h_out = h;
  return res;
}

// The W-method with Jacobian reuse (tableau ros2_w, or any other tableau taken as a W-method):
// each cell carries a cache {W, h_W, age} across attempts and calls.  An attempt of size hh reuses
// W (hence the factorisation of I/(g hh) - W) when h_W == hh and age < WAGE_MAX; otherwise it
// evaluates J at the attempt's initial state, stores it as W with h_W = hh and age 0.  Every
// accepted step ages the cache by one.  h_W <= 0 marks an empty cache.  Otherwise the controller
// of integrate_one.
constexpr int WAGE_MAX = 32;

struct WCache {
  double* W;   // N x N
  double* h;   // h_W
  int* age;
};

template <class Sys>
IntResult integrate_w(const Sys& sys, const Tableau& tb, double* y, double dt, double h_in, const IntOpts& o,
                      WCache wc, int* n_jac) {
  IntResult res;
  const int N = sys.n();
  for (int i = 0; i < N; ++i)
    if (!std::isfinite(y[i])) { res.status = NONFINITE; res.h_out = h_in; return res; }
  std::vector<double> ynew(N), e(N);
  double t = 0.0;
  double h = h_in > 0 ? h_in : dt;
  bool reject_last = false;
  for (;;) {
    if (res.attempts >= o.max_steps) { res.status = MAX_STEPS; break; }
    if (h < o.h_min) { res.status = H_UNDERFLOW; break; }
    const bool last = t + 1.0001 * h >= dt;
    const double hh = last ? dt - t : h;
    if (!(*wc.h == hh && *wc.age < WAGE_MAX)) {
      sys.jac(y, wc.W);
      *wc.h = hh;
      *wc.age = 0;
      ++*n_jac;
    }
    ros4_step(sys, tb, y, hh, ynew.data(), e.data(), wc.W);
    res.attempts++;
    double err = err_norm(N, y, ynew.data(), e.data(), o.rtol, o.atol);
    bool finite = std::isfinite(err);
    for (int i = 0; i < N && finite; ++i) finite = std::isfinite(ynew[i]);
    double fac = finite ? std::min(6.0, std::max(0.2, 0.9 * std::pow(std::max(err, 1e-10), -1.0 / tb.order))) : 0.2;
    if (finite && err <= 1.0) {
      for (int i = 0; i < N; ++i) y[i] = ynew[i];
      res.accepted++;
      ++*wc.age;
      if (reject_last) fac = std::min(fac, 1.0);
      reject_last = false;
      const double hnext = hh * fac;
      if (last) { h = hh < h ? h : hnext; break; }
      t += hh;
      h = hnext;
    } else {
      res.rejected++;
      reject_last = true;
      h = hh * fac;
    }
  }
  res.h_out = h;
  return res;
}

// Replay: the accepted step sizes of an earlier run, no error control (any scalar type).
template <class S, class Sys>
void replay(const Sys& sys, const Tableau& tb, S* y, const double* hs, int nh) {
  const int N = sys.n();
  std::vector<S> ynew(N), e(N);
  for (int s = 0; s < nh; ++s) {
    ros4_step(sys, tb, y, hs[s], ynew.data(), e.data());
    for (int i = 0; i < N; ++i) y[i] = ynew[i];
  }
}

}  // namespace orc

// ================================================================================ C interface
using namespace orc;
typedef std::complex<double> cplx;

static thread_local std::string g_err;

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void* orc_load(const char* path) {
  try {
    return new Mech(parse(path));
  } catch (const std::exception& e) {
    g_err = e.what();
    return nullptr;
  }
}

void orc_free(void* h) { delete static_cast<Mech*>(h); }

int orc_info(void* h, int* ns, int* nr, int* ne) {
  const Mech& m = *static_cast<Mech*>(h);
  *ns = m.ns; *nr = m.nr; *ne = (int)m.elements.size();
  return 0;
}

// per species: W, element counts [ne], Tmid, hf/R, s298/R
int orc_species(void* h, double* W, int* counts, double* Tmid, double* hf_R, double* s_R) {
  const Mech& m = *static_cast<Mech*>(h);
  const int ne = (int)m.elements.size();
  for (int k = 0; k < m.ns; ++k) {
    W[k] = m.sp[k].W;
    for (int e = 0; e < ne; ++e) counts[e * m.ns + k] = m.sp[k].counts[e];
    Tmid[k] = m.sp[k].Tmid; hf_R[k] = m.sp[k].hf_R; s_R[k] = m.sp[k].s_R;
  }
  return 0;
}

// reaction stoichiometry: nu_f[r][k], nu_r[r][k] (dense), kind[r], lnA[r] (SI)
int orc_reactions(void* h, int* kind, double* lnA, int* nuf, int* nur) {
  const Mech& m = *static_cast<Mech*>(h);
  for (int r = 0; r < m.nr; ++r) {
    kind[r] = m.rx[r].kind;
    lnA[r] = m.rx[r].lnA;
    for (int k = 0; k < m.ns; ++k) { nuf[r * m.ns + k] = 0; nur[r * m.ns + k] = 0; }
    for (size_t i = 0; i < m.rx[r].rsp.size(); ++i) nuf[r * m.ns + m.rx[r].rsp[i]] += m.rx[r].rnu[i];
    for (size_t i = 0; i < m.rx[r].psp.size(); ++i) nur[r * m.ns + m.rx[r].psp[i]] += m.rx[r].pnu[i];
  }
  return 0;
}

int orc_thermo(void* h, int k, double T, double* cp, double* hRT, double* sR) {
  const Mech& m = *static_cast<Mech*>(h);
  thermo(m.sp[k], T, *cp, *hRT, *sR);
  return 0;
}

int orc_thermo_cplx(void* h, int k, double Tre, double Tim, double* out /*cp,h,s re/im*/) {
  const Mech& m = *static_cast<Mech*>(h);
  cplx cp, hh, s;
  thermo(m.sp[k], cplx(Tre, Tim), cp, hh, s);
  out[0] = cp.real(); out[1] = cp.imag(); out[2] = hh.real(); out[3] = hh.imag(); out[4] = s.real(); out[5] = s.imag();
  return 0;
}

// f for n cells; y [n][Ns], P [n], lnA [Nr] or null, f [n][Ns]
int orc_source(void* h, int n, const double* y, const double* P, const double* lnA, double* f) {
  const Mech& m = *static_cast<Mech*>(h);
  for (int c = 0; c < n; ++c) source(m, y + (size_t)c * m.ns, P[c], lnA, f + (size_t)c * m.ns);
  return 0;
}

int orc_source_cplx(void* h, const double* y_re, const double* y_im, double P, const double* lnA_re,
                    const double* lnA_im, double* f_re, double* f_im) {
  const Mech& m = *static_cast<Mech*>(h);
  std::vector<cplx> y(m.ns), f(m.ns), lnA;
  for (int i = 0; i < m.ns; ++i) y[i] = cplx(y_re[i], y_im ? y_im[i] : 0.0);
  if (lnA_re) { lnA.resize(m.nr); for (int r = 0; r < m.nr; ++r) lnA[r] = cplx(lnA_re[r], lnA_im ? lnA_im[r] : 0.0); }
  source(m, y.data(), P, lnA_re ? lnA.data() : (const cplx*)nullptr, f.data());
  for (int i = 0; i < m.ns; ++i) { f_re[i] = f[i].real(); f_im[i] = f[i].imag(); }
  return 0;
}

int orc_jacobian(void* h, int n, const double* y, const double* P, const double* lnA, double* J, int nthreads) {
  const Mech& m = *static_cast<Mech*>(h);
  const size_t N = m.ns;
  std::atomic<int> next(0);
  auto work = [&]() {
    for (int c; (c = next++) < n;) jacobian(m, y + c * N, P[c], lnA, J + c * N * N);
  };
  std::vector<std::thread> th;
  for (int t = 1; t < std::max(1, nthreads); ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return 0;
}

// forward / reverse rates of progress (with [M] for THIRD) and rate constants of one cell
int orc_rates(void* h, const double* y, double P, const double* lnA, double* kf, double* kr, double* qf,
              double* qr, double* omega, double* C) {
  const Mech& m = *static_cast<Mech*>(h);
  Rates<double> R;
  rates(m, y, P, lnA, R);
  for (int r = 0; r < m.nr; ++r) { kf[r] = R.kf[r]; kr[r] = R.kr[r]; qf[r] = R.qf[r]; qr[r] = R.qr[r]; }
  for (int k = 0; k < m.ns; ++k) { omega[k] = R.omega[k]; C[k] = R.C[k]; }
  return 0;
}

// tableau `id`: s, order, gamma, a[6][6], c[6][6], m[6], e[6], explicit flag  (88 doubles)
int orc_tableau(int id, double* out) {
  Tableau t = tableau_by_id(id);
  out[87] = t.erk ? 1.0 : 0.0;
  out[0] = t.s;
  out[1] = t.order;
  out[2] = t.gamma;
  for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) { out[3 + i * 6 + j] = t.a[i][j]; out[39 + i * 6 + j] = t.c[i][j]; }
  for (int i = 0; i < 6; ++i) { out[75 + i] = t.m[i]; out[81 + i] = t.e[i]; }
  return 0;
}

// one ROS4 step on y' = A y (A n x n row-major)
int orc_step_linear(int n, const double* A, const double* y, double h, double* ynew, double* err, int tab) {
  LinSys<double> sys{n, A};
  ros4_step(sys, tableau_by_id(tab), y, h, ynew, err);
  return 0;
}

int orc_integrate_linear(int n, const double* A, double* y, double dt, double rtol, double atol, int* attempts,
                         int tab) {
  LinSys<double> sys{n, A};
  IntOpts o; o.rtol = rtol; o.atol = atol;
  IntResult r = integrate_one(sys, tableau_by_id(tab), y, dt, 0.0, o, nullptr);
  *attempts = r.attempts;
  return r.status;
}

// one ROS4 step of the chemistry of one cell
int orc_step(void* h, const double* y, double P, const double* lnA, double hstep, double* ynew, double* err, int tab) {
  const Mech& m = *static_cast<Mech*>(h);
  ChemSys<double> sys{m, P, lnA};
  ros4_step(sys, tableau_by_id(tab), y, hstep, ynew, err);
  return 0;
}

// Integrate n cells over [0, dt] in place. y [n][Ns]; h in/out (nullable, <=0 means dt);
// status/attempts/accepted/rejected per cell (nullable). Threads over cells.
int orc_integrate(void* hm, int n, double* y, const double* P, const double* lnA, double dt, double rtol,
                  double atol, double* h, int* status, int* attempts, int* accepted, int* rejected,
                  int max_steps, double h_min, double T_min, int fixed_steps, int nthreads, int tab) {
  const Mech& m = *static_cast<Mech*>(hm);
  const Tableau tb = tableau_by_id(tab);
  IntOpts o;
  o.rtol = rtol; o.atol = atol; o.max_steps = max_steps; o.h_min = h_min; o.T_min = T_min; o.fixed_steps = fixed_steps;
  std::atomic<int> next(0);
  auto work = [&]() {
    for (int c; (c = next++) < n;) {
      double* yc = y + (size_t)c * m.ns;
      IntResult r;
      if (T_min > 0 && yc[0] < T_min) {
        r.status = SKIPPED;
        r.h_out = h ? h[c] : 0.0;
      } else {
        ChemSys<double> sys{m, P[c], lnA};
        r = integrate_one(sys, tb, yc, dt, h ? h[c] : 0.0, o, nullptr);
      }
      if (h) h[c] = r.h_out;
      if (status) status[c] = r.status;
      if (attempts) attempts[c] = r.attempts;
      if (accepted) accepted[c] = r.accepted;
      if (rejected) rejected[c] = r.rejected;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < std::max(1, nthreads); ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return 0;
}

// Per-cell switching between the explicit RKF45 (tableau 4) and the Rosenbrock method `tab`
// (the policy of the GPU path's per-cell method array): method[c] > 0 = integrate with RKF45
// under at most that many attempts and, if the cell does not reach dt within them (attempt limit
// or step-size underflow), integrate it again from its initial state and step size with the
// Rosenbrock method; method[c] <= 0 = the Rosenbrock method.  Written back for the next call:
// after an explicit success with a attempts, 4a + 8; after a Rosenbrock integration with a
// attempts, 4a + 8 if dt * rho <= 3a, else 0, where rho = max_i sum_j |J_ij| w_j / w_i is the
// Gershgorin bound of the Jacobian at the initial state scaled by the error weights
// w = atol + rtol |y| (the explicit method's stability-limited steps, about dt * rho / 3, would not
// outnumber the Rosenbrock attempts).  Cells below T_min or with a non-finite state keep their
// method.  attempts and status are those of the run that finished the cell.
// alt = 5 takes the W-method (with the caches Wc, hW, age of orc_integrate_w) as the alternative:
// a cell goes to it (budget 12) after a Rosenbrock integration of one attempt whose next-step
// proposal h_out is at least 2 dt (quiescent: a cell whose single step only just fitted would
// need many steps of the second-order W-method), and every Rosenbrock integration empties the
// cell's cache.
int orc_integrate_auto(void* hm, int n, double* y, const double* P, const double* lnA, double dt, double rtol,
                       double atol, double* h, int* status, int* attempts, int* method, int max_steps,
                       double T_min, int nthreads, int tab, int alt, double* Wc, double* hW, int* wage) {
  const Mech& m = *static_cast<Mech*>(hm);
  const Tableau tr = tableau_by_id(tab), te = tableau_by_id(alt == 5 ? 5 : 4);
  std::atomic<int> next(0);
  auto work = [&]() {
    const int N = m.ns;
    std::vector<double> y0(N), J(N * N);
    for (int c; (c = next++) < n;) {
      double* yc = y + (size_t)c * N;
      const double h_in = h ? h[c] : 0.0;
      IntResult r;
      bool done = false;
      if (T_min > 0 && yc[0] < T_min) {
        r.status = SKIPPED;
        r.h_out = h_in;
        done = true;
      }
      for (int i = 0; i < N && !done; ++i)
        if (!std::isfinite(yc[i])) { r.status = NONFINITE; r.h_out = h_in; done = true; }
      ChemSys<double> sys{m, P[c], lnA};
      if (!done && method[c] > 0) {
        for (int i = 0; i < N; ++i) y0[i] = yc[i];
        IntOpts o;
        o.rtol = rtol; o.atol = atol; o.max_steps = std::min(max_steps, method[c]);
        if (alt == 5) {
          int nj = 0;
          WCache wc{Wc + (size_t)c * N * N, hW + c, wage + c};
          r = integrate_w(sys, te, yc, dt, h_in, o, wc, &nj);
        } else {
          r = integrate_one(sys, te, yc, dt, h_in, o, nullptr);
        }
        if (r.status == OK) {
          method[c] = 4 * r.attempts + 8;
          done = true;
        } else {
          for (int i = 0; i < N; ++i) yc[i] = y0[i];
        }
      }
      if (!done) {
        sys.jac(yc, J.data());
        double rho = 0.0;
        for (int i = 0; i < N; ++i) {
          double sum = 0.0;
          for (int j = 0; j < N; ++j) sum += std::fabs(J[i * N + j]) * (atol + rtol * std::fabs(yc[j]));
          rho = std::max(rho, sum / (atol + rtol * std::fabs(yc[i])));
        }
        IntOpts o;
        o.rtol = rtol; o.atol = atol; o.max_steps = max_steps;
        r = integrate_one(sys, tr, yc, dt, h_in, o, nullptr);
        if (alt == 5) {
          method[c] = (r.status == OK && r.attempts == 1 && r.h_out >= 2.0 * dt) ? 12 : 0;
          hW[c] = 0.0;
        } else {
          method[c] = (r.status == OK && dt * rho <= 3.0 * r.attempts) ? 4 * r.attempts + 8 : 0;
        }
      }
      if (h) h[c] = r.h_out;
      if (status) status[c] = r.status;
      if (attempts) attempts[c] = r.attempts;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < std::max(1, nthreads); ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return 0;
}

// The W-method with Jacobian reuse over n cells (see integrate_w); the caches Wc [n x N x N],
// hW [n] and age [n] persist between calls (zero hW to empty them); n_jac [n] out: Jacobian
// evaluations of this call.
int orc_integrate_w(void* hm, int n, double* y, const double* P, const double* lnA, double dt, double rtol,
                    double atol, double* h, int* status, int* attempts, int* n_jac, double* Wc, double* hW,
                    int* age, int max_steps, int nthreads, int tab) {
  const Mech& m = *static_cast<Mech*>(hm);
  const Tableau tb = tableau_by_id(tab);
  IntOpts o;
  o.rtol = rtol; o.atol = atol; o.max_steps = max_steps;
  std::atomic<int> next(0);
  auto work = [&]() {
    const int N = m.ns;
    for (int c; (c = next++) < n;) {
      ChemSys<double> sys{m, P[c], lnA};
      int nj = 0;
      WCache wc{Wc + (size_t)c * N * N, hW + c, age + c};
      IntResult r = integrate_w(sys, tb, y + (size_t)c * N, dt, h ? h[c] : 0.0, o, wc, &nj);
      if (h) h[c] = r.h_out;
      if (status) status[c] = r.status;
      if (attempts) attempts[c] = r.attempts;
      if (n_jac) n_jac[c] = nj;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < std::max(1, nthreads); ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return 0;
}

// One step of size h of the method `tab` with the matrix W (N x N) in place of the Jacobian.
int orc_step_w(void* hm, const double* y, double P, const double* lnA, double h, const double* W, double* ynew,
               double* err, int tab) {
  const Mech& m = *static_cast<Mech*>(hm);
  ChemSys<double> sys{m, P, lnA};
  ros4_step(sys, tableau_by_id(tab), y, h, ynew, err, W);
  return 0;
}

// One cell, recording the accepted step sizes (hs capacity cap; returns count or -1).
int orc_integrate_log(void* hm, double* y, double P, const double* lnA, double dt, double rtol, double atol,
                      double h_in, int max_steps, double* hs, int cap, int* status, double* h_out) {
  const Mech& m = *static_cast<Mech*>(hm);
  IntOpts o;
  o.rtol = rtol; o.atol = atol; o.max_steps = max_steps;
  std::vector<double> acc;
  ChemSys<double> sys{m, P, lnA};
  IntResult r = integrate_one(sys, ros4_hw(), y, dt, h_in, o, &acc);
  *status = r.status;
  *h_out = r.h_out;
  if ((int)acc.size() > cap) return -1;
  for (size_t i = 0; i < acc.size(); ++i) hs[i] = acc[i];
  return (int)acc.size();
}

// Replay a fixed step sequence in complex arithmetic (complex-step sensitivities).
int orc_replay_cplx(void* hm, double* y_re, double* y_im, double P, const double* lnA_re, const double* lnA_im,
                    const double* hs, int nh) {
  const Mech& m = *static_cast<Mech*>(hm);
  std::vector<cplx> y(m.ns), lnA;
  for (int i = 0; i < m.ns; ++i) y[i] = cplx(y_re[i], y_im[i]);
  if (lnA_re) { lnA.resize(m.nr); for (int r = 0; r < m.nr; ++r) lnA[r] = cplx(lnA_re[r], lnA_im ? lnA_im[r] : 0.0); }
  ChemSys<cplx> sys{m, P, lnA_re ? lnA.data() : (const cplx*)nullptr};
  replay(sys, ros4_hw(), y.data(), hs, nh);
  for (int i = 0; i < m.ns; ++i) { y_re[i] = y[i].real(); y_im[i] = y[i].imag(); }
  return 0;
}

// Replay in double (the forward map of a frozen step sequence).
int orc_replay(void* hm, double* y, double P, const double* lnA, const double* hs, int nh) {
  const Mech& m = *static_cast<Mech*>(hm);
  ChemSys<double> sys{m, P, lnA};
  replay(sys, ros4_hw(), y, hs, nh);
  return 0;
}

}  // extern "C"
