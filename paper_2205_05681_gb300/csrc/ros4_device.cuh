// Device code of the batched ROS4 chemistry integrator (FP64, sm_103a).
//
// Compiled at run time by NVRTC, once per mechanism and launch configuration, after a
// generated header (chem_host.cpp, emit_mechanism) that defines:
//   NS, NR            species and reactions; the state length is NS ([T, n_1..n_{NS-1}])
//   TEAM, TPB         lanes per cell (1, 32 or TPB) and threads per block
//   MAXP              largest number of distinct species on one side of a reaction
//   tables mk_*       NASA-7 coefficients pre-divided for cp, h and s; Arrhenius data; species
//                     lists; efficiencies; falloff data (see emit_mechanism)
//
// What the kernels compute (Curtis, Niemeyer & Sung):
//   * f(y), Sec. 2.1 Eq. (e:dphidt): concentrations from the unit-mass closure of Eq. (e:n_nsp);
//     NASA-7 thermo; Arrhenius / third-body / Lindemann / Troe forward rates; reverse rates from
//     the equilibrium constant; net production rates; dT/dt from the constant-pressure energy
//     balance;
//   * the analytical Jacobian J = df/dy, Eq. (e:jac), in closed form: the reaction part
//     d(omega)/dC (sparse scatter plus the dense third-body efficiency part), then the chain
//     rule to the [T, n] state (the bath-gas column, the volume terms and the temperature row);
//   * the transformed ROS4 step of Sec. 2.3 with partial-pivoting LU of (I/(gamma h) - J), four
//     stage solves (three f evaluations: the Hairer-Wanner set repeats stage 3's argument for
//     stage 4), the embedded error estimate and the step-size controller;
//   * batching (Sec. 2.4.1): a persistent kernel whose teams pull cells from a device work
//     queue, and a plain form that runs one step attempt per launch.
//
// Work decomposition.  A "team" of TEAM threads owns one cell at a time; all of the cell's
// working set (the N x N matrix, stage vectors, thermo and rate scratch) sits in shared memory.
// TEAM == 1: one thread per cell, arrays interleaved across the block's threads (stride TPB)
// so that lane-consecutive accesses hit consecutive banks.  TEAM == 4, 8, 16: several cells per
// warp (sub-warp teams, for small mechanisms whose loops would leave most lanes of a wider team
// idle), contiguous arrays per team, team-masked warp synchronisation and shuffles.  TEAM == 32:
// a warp per cell.  TEAM == TPB (64..256): a block per cell.  Reaction loops give each lane a
// subset of reactions and scatter into the shared Jacobian with shared-memory atomics (TEAM>1).
// Every device loop is bounded; there is no grid-wide wait.

#define ELEM 0
#define THIRD 1
#define LIND 2
#define TROE 3

#define R_U 8314.462618
#define INV_R_U (1.0 / 8314.462618)
#define P_ATM 101325.0
#define R_OVER_PATM (8314.462618 / 101325.0)
#define PATM_OVER_R (101325.0 / 8314.462618)
#define LN10 2.302585092994046

#define ST_OK 0
#define ST_MAX_STEPS 1
#define ST_H_UNDERFLOW 2
#define ST_NONFINITE 3
#define ST_SKIPPED 4
#define ST_TAPE_FULL 5

#define NEQ NS
#define NB ((NEQ + WL - 1) / WL)  // WL-row chunks of a state vector held by the first warp
#define BATH (NS - 1)

#define SUBWARP (TEAM > 1 && TEAM < 32)
#if TEAM == 1
#define SS TPB
#define NTEAM TPB
#elif TEAM <= 32
#define SS 1
#define NTEAM (TPB / TEAM)
#else
#define SS 1
#define NTEAM 1
#endif
// lanes of the team's first warp (the warp-level parts: pivot scale, stage solves) and the
// first butterfly offset of a team reduction
#define WL (TEAM < 32 ? TEAM : 32)
#define XOR0 (WL / 2)

// per-cell shared-memory slots (units of SS doubles), sized so that eight 53-species cells fit
// in one SM's shared memory:
// * f at a stage argument overwrites the argument (OFF_F = OFF_YT): the argument is dead once
//   the concentrations and thermo are formed from it;
// * the three per-species arrays only the Jacobian assembly uses alias YT, U2, U3, which are
//   dead while the Jacobian is formed (it is the first thing a step attempt computes); the
//   chain rule writes JT over DOMT and BE over BK in place;
// * the LU keeps 1/U_kk on the diagonal of A, and the row permutation is packed two ints per
//   slot (the single-lane layout also keeps the pivot sequence).
#define OFF_A 0
#define OFF_Y (OFF_A + NEQ * NEQ)
#define OFF_U1 (OFF_Y + NEQ)
#define OFF_YT (OFF_U1 + NEQ)
#define OFF_F OFF_YT
#define OFF_U2 (OFF_YT + NEQ)
#define OFF_U3 (OFF_U2 + NEQ)
#define OFF_U4 (OFF_U3 + NEQ)
// at least three stage slots after the stage argument (YT, U2, U3): the Jacobian assembly's
// three per-species arrays alias them (a two-stage method has no U3 of its own)
#define NSTG (RS > 3 ? RS : 3)
#if NEED_F0
#define OFF_F0 (OFF_U2 + (NSTG - 1) * NEQ)  // f(y) kept for a later stage whose argument is y itself
#define OFF_C (OFF_F0 + NEQ)
#else
#define OFF_C (OFF_U2 + (NSTG - 1) * NEQ)
#endif
#define OFF_CP (OFF_C + NS)
#define OFF_HRT (OFF_CP + NS)
#define OFF_EX (OFF_HRT + NS)
#define OFF_IEX (OFF_EX + NS)
#define OFF_OM (OFF_IEX + NS)
#define OFF_DOMT OFF_YT
#define OFF_BK (OFF_DOMT + NS)
#define OFF_AL (OFF_BK + NS)
#define OFF_JT OFF_DOMT
#define OFF_BE OFF_BK
#define PACKED_INTS(n) (((n) + 1) / 2)
#if TEAM == 1
#define OFF_PIV (OFF_OM + NS)
#define OFF_PERM (OFF_PIV + PACKED_INTS(NEQ))
#else
#define OFF_PERM (OFF_OM + NS)
#endif
#define OFF_RED (OFF_PERM + PACKED_INTS(NEQ))
#define SLOTS (OFF_RED + 24)
// distance between consecutive teams' slots: for sub-warp teams padded to TEAM (mod 16) doubles,
// so that the teams of a half-warp reading the same offset of their arrays use disjoint banks
#if SUBWARP
#define TSTRIDE (SLOTS + ((TEAM - SLOTS % 16 + 16) % 16))
#else
#define TSTRIDE SLOTS
#endif
#define UOFF(i) ((i) == 0 ? OFF_U1 : OFF_U2 + ((i) - 1) * NEQ)

// Per-cell cache of the W-method's factorised iteration matrix (chem_int_opts.jac_cache, global
// memory, one contiguous block per cell whatever the launch configuration): the N x N factors with
// 1/U_kk on the diagonal, the composed row permutation and the pivot sequence (packed ints), the
// step size h_W they were built for (0: empty) and their age in accepted steps.  A new factorisation
// (Jacobian at the attempt's state) is made when h_W differs from the attempt's step size or
// the age reaches WAGE_MAX.
#define WC_PERM (NEQ * NEQ)
#define WC_PIV (WC_PERM + PACKED_INTS(NEQ))
#define WC_H (WC_PIV + PACKED_INTS(NEQ))
#define WC_AGE (WC_H + 1)
#define WC_STRIDE (WC_AGE + 1)
#define WAGE_MAX 32

// ------------------------------------------------------------------------------ team plumbing

// mask of the calling lane's team within its warp (all lanes for TEAM >= 32)
__device__ __forceinline__ unsigned team_mask() {
#if SUBWARP
  return ((1u << TEAM) - 1u) << ((threadIdx.x & 31) & ~(TEAM - 1));
#else
  return 0xffffffffu;
#endif
}

__device__ __forceinline__ void tsync() {
#if SUBWARP
  __syncwarp(team_mask());
#elif TEAM == 32
  __syncwarp();
#elif TEAM > 32
  __syncthreads();
#endif
}

struct Team {
  double* base;  // element i of array at slot offset o: base[(o + i) * SS]
  int tl;        // lane within the team
  __device__ __forceinline__ double& at(int o, int i) const { return base[(o + i) * SS]; }
  __device__ __forceinline__ double& A(int i, int j) const { return base[(OFF_A + i * NEQ + j) * SS]; }
#if TEAM == 1
  __device__ __forceinline__ int& piv(int i) const {
    return reinterpret_cast<int*>(&base[(OFF_PIV + (i >> 1)) * SS])[i & 1];
  }
#endif
  __device__ __forceinline__ int& perm(int i) const {
    return reinterpret_cast<int*>(&base[(OFF_PERM + (i >> 1)) * SS])[i & 1];
  }
  // 1/U_kk of the factorised matrix, kept on its diagonal
  __device__ __forceinline__ double& invd(int k) const { return A(k, k); }
};

// sum over the team; every lane gets the same bits (butterfly with commutative adds)
__device__ __forceinline__ double team_sum(const Team& tm, double v) {
#if TEAM == 1
  return v;
#else
  const unsigned msk = team_mask();
#pragma unroll
  for (int o = XOR0; o > 0; o >>= 1) v += __shfl_xor_sync(msk, v, o);
#if TEAM > 32
  double* red = &tm.base[OFF_RED];
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = 0.0;
  for (int w = 0; w < TEAM / 32; ++w) v += red[w];
  __syncthreads();
#endif
  return v;
#endif
}

// maximum over the team (same reduction tree as team_sum)
__device__ __forceinline__ double team_max(const Team& tm, double v) {
#if TEAM == 1
  return v;
#else
  const unsigned msk = team_mask();
#pragma unroll
  for (int o = XOR0; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(msk, v, o));
#if TEAM > 32
  double* red = &tm.base[OFF_RED];
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = red[0];
  for (int w = 1; w < TEAM / 32; ++w) v = fmax(v, red[w]);
  __syncthreads();
#endif
  return v;
#endif
}

// any-lane flag over the team
__device__ __forceinline__ bool team_any(const Team& tm, bool f) {
#if TEAM == 1
  return f;
#elif TEAM <= 32
  return __any_sync(team_mask(), f);
#else
  return __syncthreads_or(f) != 0;
#endif
}

template <class T>
__device__ __forceinline__ void scatter_add(double* p, double v) {
#if TEAM == 1
  *p += v;
#else
  atomicAdd(p, v);
#endif
}

// |x| as an order-preserving integer (integer pipe instead of the FP64 pipe)
__device__ __forceinline__ long long abs_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

// ------------------------------------------------------------------------------ thermo + C

// Concentrations, thermo per species and mixture sums for state y (slot OFF_Y or OFF_YT).
// Returns V; writes C, cp, h/RT, exp(s/R - h/RT), its inverse and (WJ) dcp/dT.
struct CellScalars {
  double T, invT, lnT, V, cpm, dcpm;  // cpm = sum n_k cp_k / R, dcpm = sum n_k dcp_k/dT / R
};

// mass closure: n_bath = (1 - sum_k W_k n_k) / W_bath; n_tot = sum of all moles; V = n_tot R T/P
__device__ __forceinline__ void closure_scalars(double T, double P, double wsum, double nsum, double* out) {
  const double nb = (1.0 - wsum) * mk_invW[BATH];
  const double V = (nsum + nb) * R_U * T / P;
  out[0] = 1.0 / T;
  out[1] = log(T);
  out[2] = nb;
  out[3] = V;
  out[4] = 1.0 / V;
}

template <bool WJ>
__device__ __forceinline__ void thermo_conc(const Team& tm, int oy, double P, CellScalars& cs) {
  const double T = tm.at(oy, 0);
  double sc[5];
#if TEAM > 32
  // one lane computes the cell's scalars (divisions, log) and shares them: every extra warp
  // repeating them would pay full warp-level FP64 pipe time
  if (tm.tl < 32) {
    double wsum = 0.0, nsum = 0.0;
    for (int k = tm.tl; k < NS - 1; k += 32) {
      const double n = tm.at(oy, 1 + k);
      wsum += mk_W[k] * n;
      nsum += n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
      nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
    }
    if (tm.tl == 0) {
      closure_scalars(T, P, wsum, nsum, sc);
      for (int i = 0; i < 5; ++i) tm.base[OFF_RED + 16 + i] = sc[i];
    }
  }
  __syncthreads();
  for (int i = 0; i < 5; ++i) sc[i] = tm.base[OFF_RED + 16 + i];
#else
  double wsum = 0.0, nsum = 0.0;
  for (int k = tm.tl; k < NS - 1; k += TEAM) {
    const double n = tm.at(oy, 1 + k);
    wsum += mk_W[k] * n;
    nsum += n;
  }
  wsum = team_sum(tm, wsum);
  nsum = team_sum(tm, nsum);
  closure_scalars(T, P, wsum, nsum, sc);
#endif
  const double invT = sc[0], lnT = sc[1], nb = sc[2], V = sc[3], invV = sc[4];
  double cpm = 0.0, dcpm = 0.0;
  for (int k = tm.tl; k < NS; k += TEAM) {
    const double n = k < NS - 1 ? tm.at(oy, 1 + k) : nb;
    tm.at(OFF_C, k) = n * invV;
    const int r = T < mk_Tmid[k] ? 0 : 1;
    const double* c = mk_cp[k][r];
    const double* hh = mk_h[k][r];
    const double* s = mk_s[k][r];
    const double cp = c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
    const double hRT = hh[0] + T * (hh[1] + T * (hh[2] + T * (hh[3] + T * hh[4]))) + hh[5] * invT;
    const double sR = s[0] * lnT + s[6] + T * (s[1] + T * (s[2] + T * (s[3] + T * s[4])));
    tm.at(OFF_CP, k) = cp;
    tm.at(OFF_HRT, k) = hRT;
    const double ex = exp(sR - hRT);
    tm.at(OFF_EX, k) = ex;
    tm.at(OFF_IEX, k) = 1.0 / ex;
    cpm += n * cp;
    if (WJ) {
      const double* d = mk_dcp[k][r];
      const double dcp = d[0] + T * (d[1] + T * (d[2] + T * d[3]));
      dcpm += n * dcp;
    }
  }
  cs.T = T;
  cs.invT = invT;
  cs.lnT = lnT;
  cs.V = V;
  cs.cpm = team_sum(tm, cpm);
  if (WJ) cs.dcpm = team_sum(tm, dcpm);
  tsync();
}

// ------------------------------------------------------------------------------ reactions

// -x by flipping the sign bit (integer pipe)
__device__ __forceinline__ double dneg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}
// nu * x for an integer stoichiometric coefficient nu (nuf = nu as a double): no FP64
// instruction when |nu| = 1, the common case.  The adjoint module keeps the multiply (its
// kernels measured faster with it); the results are the same bits either way.
__device__ __forceinline__ double nu_times(int nu, double nuf, double x) {
#if defined(CHEM_ADJOINT)
  return nuf * x;
#else
  if (nu == 1) return x;
  if (nu == -1) return dneg(x);
  return nuf * x;
#endif
}

// species index -> row/column of the state matrix: species 0..NS-2 -> 1..NS-1, bath -> 0
__device__ __forceinline__ int smap(int k) { return k == BATH ? 0 : k + 1; }

// Net production rates omega (slot OFF_OM, zeroed by the caller) and, with WJ, the reaction
// part of the Jacobian: A[smap(k)][smap(j)] += d omega_k / d C_j (without the default-
// efficiency third-body part, which is collected per species in OFF_BK), d omega_k/dT at
// constant C in OFF_DOMT.  The caller zeroes A, OFF_DOMT and OFF_BK.
template <bool WJ>
__device__ __forceinline__ void reaction_loop(const Team& tm, const CellScalars& cs, double P,
                                              const double* __restrict__ lnA_ext) {
  const double T = cs.T, invT = cs.invT, lnT = cs.lnT;
  const double Ctot = P * invT * INV_R_U;    // sum_k C_k = P / (R T)
  const double rtp = R_OVER_PATM * T;       // (P_atm / R T)^-1
  const double irtp = PATM_OVER_R * invT;
  for (int r = tm.tl; r < NR; r += TEAM) {
    const int kind = mk_kind[r];
    const double lA = lnA_ext ? lnA_ext[mk_rorig[r]] : mk_lnA[r];
    const double kinf = exp(lA + mk_b[r] * lnT - mk_th[r] * invT);
    double kf = kinf;
    double dlkf_dT = 0.0, dlkf_dM = 0.0;
    double M = 0.0;
    if (WJ) dlkf_dT = (mk_b[r] + mk_th[r] * invT) * invT;
    if (kind != ELEM) {
      M = Ctot;
      for (int e = mk_effoff[r]; e < mk_effoff[r + 1]; ++e) M += mk_effval[e] * tm.at(OFF_C, mk_effsp[e]);
    }
    if (kind >= LIND) {
      const double k0 = exp(mk_lnA0[r] + mk_b0[r] * lnT - mk_th0[r] * invT);
      double Pr = k0 * M / kinf;
      bool floored = false;
      if (Pr < 1e-300) { Pr = 1e-300; floored = true; }
      double F = 1.0, dlF_dlPr = 0.0, dlF_dT = 0.0;
      if (kind == TROE) {
        const double a = mk_troe[r][0];
        const double e3 = exp(-T * mk_troe[r][1]);
        const double e1 = exp(-T * mk_troe[r][2]);
        const double T2 = mk_troe[r][3];
        const double e2 = T2 > 0.0 ? exp(-T2 * invT) : 0.0;
        const double Fc = (1.0 - a) * e3 + a * e1 + e2;
        const double lFc = log10(Fc);
        const double c = -0.4 - 0.67 * lFc;
        const double n = 0.75 - 1.27 * lFc;
        const double x = log10(Pr) + c;
        const double d = n - 0.14 * x;
        const double id = 1.0 / d;
        const double f1 = x * id;
        const double den = 1.0 / (1.0 + f1 * f1);
        const double lF = lFc * den;
        F = exp(lF * LN10);
        if (WJ) {
          const double g2 = 2.0 * lFc * f1 * den * den;  // -d log10F / d f1
          if (!floored) dlF_dlPr = -g2 * n * id * id;
          const double dFc = -(1.0 - a) * mk_troe[r][1] * e3 - a * mk_troe[r][2] * e1 +
                             (T2 > 0.0 ? T2 * invT * invT * e2 : 0.0);
          const double df1_dlFc = (-0.67 * n + 1.27 * x) * id * id;
          const double dlog10F_dlFc = den - g2 * df1_dlFc;
          dlF_dT = dlog10F_dlFc * dFc / Fc;
        }
      }
      kf = kinf * (Pr / (1.0 + Pr)) * F;
      if (WJ) {
        const double g = floored ? 0.0 : 1.0 / (1.0 + Pr) + dlF_dlPr;
        const double dlk0 = (mk_b0[r] + mk_th0[r] * invT) * invT;
        dlkf_dM = g / M;
        dlkf_dT = dlkf_dT + g * (dlk0 - dlkf_dT) + dlF_dT;
      }
    }
    // reverse constant: k_r = k_f / K_c with K_c = prod exp(s/R - h/RT)^nu (P_atm/RT)^dnu
    double kr = kf;
    double fwd = kf;
    const int nre = mk_nre[r], npr = mk_npr[r];
    for (int i = 0; i < nre; ++i) {
      const int sp = mk_rsp[r][i];
      const double c = tm.at(OFF_C, sp), ex = tm.at(OFF_EX, sp);
      for (int v = 0; v < mk_rnu[r][i]; ++v) { fwd *= c; kr *= ex; }
    }
    double rev = 1.0;
    for (int i = 0; i < npr; ++i) {
      const int sp = mk_psp[r][i];
      const double c = tm.at(OFF_C, sp), iex = tm.at(OFF_IEX, sp);
      for (int v = 0; v < mk_pnu[r][i]; ++v) { rev *= c; kr *= iex; }
    }
    const int dnu = mk_dnu[r];
    for (int v = 0; v < dnu; ++v) kr *= rtp;
    for (int v = 0; v < -dnu; ++v) kr *= irtp;
    rev *= kr;
    const double m = kind == THIRD ? M : 1.0;
    const double qnet = fwd - rev;
    const double q = m * qnet;
    // shared-memory reductions without a return value do not stall the lane (TEAM > 1)
    for (int i = 0; i < nre; ++i)
      scatter_add<double>(&tm.at(OFF_OM, mk_rsp[r][i]), nu_times(-mk_rnu[r][i], -mk_rnuf[r][i], q));
    for (int i = 0; i < npr; ++i)
      scatter_add<double>(&tm.at(OFF_OM, mk_psp[r][i]), nu_times(mk_pnu[r][i], mk_pnuf[r][i], q));
    if (WJ) {
      // d ln Kc / dT = (sum nu'' h/RT - sum nu' h/RT - dnu) / T
      double dlKc = -mk_dnuf[r];
      for (int i = 0; i < npr; ++i) dlKc += mk_pnuf[r][i] * tm.at(OFF_HRT, mk_psp[r][i]);
      for (int i = 0; i < nre; ++i) dlKc -= mk_rnuf[r][i] * tm.at(OFF_HRT, mk_rsp[r][i]);
      dlKc *= invT;
      const double dqdT = m * (fwd * dlkf_dT - rev * (dlkf_dT - dlKc));
      // dq/d[M]: the [M] factor of THIRD reactions, the falloff blend of LIND/TROE
      const double beta = kind == THIRD ? qnet : (kind == ELEM ? 0.0 : qnet * dlkf_dM);
      // dq/dC_j of the mass-action products
      double dq[2 * MAXP];
      int dsp[2 * MAXP];
      int nd = 0;
      for (int i = 0; i < nre; ++i) {
        const int nu = mk_rnu[r][i];
        double p = m * kf * mk_rnuf[r][i];
        for (int i2 = 0; i2 < nre; ++i2) {
          const double c = tm.at(OFF_C, mk_rsp[r][i2]);
          const int e = i2 == i ? nu - 1 : mk_rnu[r][i2];
          for (int v = 0; v < e; ++v) p *= c;
        }
        dq[nd] = p;
        dsp[nd++] = mk_rsp[r][i];
      }
      for (int i = 0; i < npr; ++i) {
        const int nu = mk_pnu[r][i];
        double p = -m * kr * mk_pnuf[r][i];
        for (int i2 = 0; i2 < npr; ++i2) {
          const double c = tm.at(OFF_C, mk_psp[r][i2]);
          const int e = i2 == i ? nu - 1 : mk_pnu[r][i2];
          for (int v = 0; v < e; ++v) p *= c;
        }
        dq[nd] = p;
        dsp[nd++] = mk_psp[r][i];
      }
      for (int side = 0; side < 2; ++side) {
        const int np = side == 0 ? nre : npr;
        for (int i = 0; i < np; ++i) {
          const int k = side == 0 ? mk_rsp[r][i] : mk_psp[r][i];
          const int nui = side == 0 ? -mk_rnu[r][i] : mk_pnu[r][i];
          const double nuk = side == 0 ? -mk_rnuf[r][i] : mk_pnuf[r][i];
          const int row = smap(k);
          for (int d = 0; d < nd; ++d) scatter_add<double>(&tm.A(row, smap(dsp[d])), nu_times(nui, nuk, dq[d]));
          scatter_add<double>(&tm.at(OFF_DOMT, k), nu_times(nui, nuk, dqdT));
          if (kind != ELEM) {
            const double nb = nu_times(nui, nuk, beta);
            scatter_add<double>(&tm.at(OFF_BK, k), nb);
            for (int e = mk_effoff[r]; e < mk_effoff[r + 1]; ++e)
              scatter_add<double>(&tm.A(row, smap(mk_effsp[e])), nb * mk_effval[e]);
          }
        }
      }
    }
  }
  tsync();
}

// f from omega: f[0] = dT/dt = -T sum_k (h_k/RT) V omega_k / sum_k n_k cp_k/R,
// f[1+k] = V omega_k.  Returns dT/dt.
__device__ __forceinline__ double source_from_omega(const Team& tm, const CellScalars& cs, int of) {
  double hs = 0.0;
  for (int k = tm.tl; k < NS; k += TEAM) {
    const double om = tm.at(OFF_OM, k);
    hs += tm.at(OFF_HRT, k) * om;
    if (k < NS - 1) tm.at(of, 1 + k) = cs.V * om;
  }
  hs = team_sum(tm, hs);
  const double fT = -cs.T * cs.V * hs / cs.cpm;
  if (tm.tl == 0) tm.at(of, 0) = fT;
  tsync();
  return fT;
}

__device__ __forceinline__ void zero_rates(const Team& tm, bool with_j) {
  for (int k = tm.tl; k < NS; k += TEAM) {
    tm.at(OFF_OM, k) = 0.0;
    if (with_j) { tm.at(OFF_DOMT, k) = 0.0; tm.at(OFF_BK, k) = 0.0; }
  }
  if (with_j)
    for (int e = tm.tl; e < NEQ * NEQ; e += TEAM) tm.at(OFF_A, e) = 0.0;
  tsync();
}

// f(y) into slot `of` for the state at slot `oy`.
__device__ void eval_f(const Team& tm, int oy, int of, double P, const double* lnA_ext) {
  CellScalars cs;
  thermo_conc<false>(tm, oy, P, cs);
  zero_rates(tm, false);
  reaction_loop<false>(tm, cs, P, lnA_ext);
  source_from_omega(tm, cs, of);
}

// f(y) into `of` and the state Jacobian into A: A = sgn * J + shift * I.
// sgn = +1, shift = 0 gives J; sgn = -1, shift = 1/(gamma h) gives M = I/(gamma h) - J.
__device__ void eval_f_jac(const Team& tm, int oy, int of, double P, const double* lnA_ext,
                           double sgn, double shift) {
  CellScalars cs;
  thermo_conc<true>(tm, oy, P, cs);
  zero_rates(tm, true);
  reaction_loop<true>(tm, cs, P, lnA_ext);
  const double fT = source_from_omega(tm, cs, of);
  const double T = cs.T, V = cs.V, invT = cs.invT;
  const double Ctot = P * invT * INV_R_U;
  const double RTP = 1.0 / Ctot;  // R T / P
  // per species row k (B_k = default-efficiency third-body part, added to every column):
  //   D_k = omega_k - sum_m (d omega_k/dC_m) C_m,
  //   d f_k/d n_j = d omega_k/dC_j - w_j d omega_k/dC_bath + (RT/P)(1 - w_j) D_k
  //               = A_kj + P1_k - w_j P2_k with P1 = B_k + (RT/P) D_k, P2 = A_kb + B_k + (RT/P) D_k,
  //   d f_k / dT = V (D_k / T + d omega_k/dT).
  for (int k = tm.tl; k < NS; k += TEAM) {
    const int row = smap(k);
    // four partial sums: independent FMA chains instead of one NS-long dependent chain
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    int j = 0;
    for (; j + 3 < NS; j += 4) {
      d0 += tm.A(row, smap(j)) * tm.at(OFF_C, j);
      d1 += tm.A(row, smap(j + 1)) * tm.at(OFF_C, j + 1);
      d2 += tm.A(row, smap(j + 2)) * tm.at(OFF_C, j + 2);
      d3 += tm.A(row, smap(j + 3)) * tm.at(OFF_C, j + 3);
    }
    for (; j < NS; ++j) d0 += tm.A(row, smap(j)) * tm.at(OFF_C, j);
    const double dot = (d0 + d1) + (d2 + d3);
    const double Bk = tm.at(OFF_BK, k);
    const double D = tm.at(OFF_OM, k) - dot - Bk * Ctot;
    tm.at(OFF_AL, k) = tm.A(row, 0) + Bk + RTP * D;
    tm.at(OFF_BE, k) = Bk + RTP * D;
    tm.at(OFF_JT, k) = V * (D * invT + tm.at(OFF_DOMT, k));
  }
  tsync();
  // species rows, w_j = W_j / W_bath
#if TEAM == 1
  for (int i = 1; i < NEQ; ++i) {
    const int k = i - 1;
    const double al = tm.at(OFF_AL, k), be = tm.at(OFF_BE, k);
    for (int l = 1; l < NEQ; ++l) {
      const double w = mk_wratio[l - 1];
      const double J = tm.A(i, l) - w * al + be;
      tm.A(i, l) = sgn * J + (i == l ? shift : 0.0);
    }
    tm.A(i, 0) = sgn * tm.at(OFF_JT, k);
  }
#else
  for (int e = tm.tl; e < (NEQ - 1) * NEQ; e += TEAM) {
    const int i = 1 + e / NEQ, l = e - (i - 1) * NEQ;
    const int k = i - 1;
    if (l == 0) {
      tm.A(i, 0) = sgn * tm.at(OFF_JT, k);
    } else {
      const double w = mk_wratio[l - 1];
      const double J = tm.A(i, l) - w * tm.at(OFF_AL, k) + tm.at(OFF_BE, k);
      tm.A(i, l) = sgn * J + (i == l ? shift : 0.0);
    }
  }
#endif
  tsync();
  // temperature row: f_T = -Q / cpm with Q = T sum_k (h_k/RT) f'_k over all species (f'_k =
  // V omega_k, bath included); dQ/dn_j = T sum_k (h_k/RT) J_kj, dQ/dT = sum_k cp_k f'_k +
  // T sum_k (h_k/RT) J_kT; d cpm/dn_j = cp_j - w_j cp_bath, d cpm/dT = sum_k n_k dcp_k/dT.
  const double hb = tm.at(OFF_HRT, BATH), alb = tm.at(OFF_AL, BATH), beb = tm.at(OFF_BE, BATH);
  const double icpm = 1.0 / cs.cpm;
  double cpf = 0.0;  // sum_k cp_k omega_k, a team reduction rather than one lane's loop
  for (int k = tm.tl; k < NS; k += TEAM) cpf += tm.at(OFF_CP, k) * tm.at(OFF_OM, k);
  cpf = team_sum(tm, cpf);
  for (int l = tm.tl; l < NEQ; l += TEAM) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 1;
    for (; i + 3 < NEQ; i += 4) {
      s0 += tm.at(OFF_HRT, i - 1) * tm.A(i, l);
      s1 += tm.at(OFF_HRT, i) * tm.A(i + 1, l);
      s2 += tm.at(OFF_HRT, i + 1) * tm.A(i + 2, l);
      s3 += tm.at(OFF_HRT, i + 2) * tm.A(i + 3, l);
    }
    for (; i < NEQ; ++i) s0 += tm.at(OFF_HRT, i - 1) * tm.A(i, l);
    double s = (s0 + s1) + (s2 + s3);
    if (l > 0) s -= tm.at(OFF_HRT, l - 1) * shift;  // remove the diagonal shift of M
    s *= sgn;  // the rows above carry the sign
    double val;
    if (l == 0) {
      s += hb * tm.at(OFF_JT, BATH);
      const double dQdT = cpf * V + T * s;
      val = -(dQdT + fT * cs.dcpm) * icpm;
    } else {
      const double w = mk_wratio[l - 1];
      const double Jb = tm.A(0, l) - w * alb + beb;  // bath row, before it is overwritten
      s += hb * Jb;
      const double dcpm = tm.at(OFF_CP, l - 1) - w * tm.at(OFF_CP, BATH);
      val = -(T * s + fT * dcpm) * icpm;
    }
    tm.A(0, l) = sgn * val + (l == 0 ? shift : 0.0);
  }
  tsync();
}

// ------------------------------------------------------------------------------ LU + solves

#if TEAM >= 128
// Look-ahead part of the multi-warp LU, run by the team's first warp: column c (rows c..N-1)
// receives the rank-1 update of step c-1 (c > 0), then its pivot (largest |a|, lowest row on
// ties) and the pivot's inverse go to the team's scratch slots LU_PIV / LU_INV.
#define LU_INV (OFF_RED + 21)
#define LU_PIV (OFF_RED + 22)
__device__ __forceinline__ void lu_panel(const Team& tm, int c) {
  long long best = -1;
  int p = NEQ;
  const double u = c > 0 ? tm.A(c - 1, c) : 0.0;
  for (int i = c + tm.tl; i < NEQ; i += 32) {
    double a = tm.A(i, c);
    if (c > 0) {
      a = fma(-tm.A(i, c - 1), u, a);
      tm.A(i, c) = a;
    }
    const long long v = abs_key(a);
    if (v > best) { best = v; p = i; }
  }
  {
    // warp argmax in three reductions: the high word of the key, the low word among the lanes
    // holding that maximum, the lowest row among the lanes holding both (a lane without rows
    // enters key 0 with row NEQ and so never wins over a row of the column)
    const unsigned long long key = best < 0 ? 0ULL : (unsigned long long)best;
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    p = (int)__reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? (unsigned)p : 0xffffffffu);
  }
  __syncwarp();  // the updated column is visible to the whole warp
  const double inv = 1.0 / tm.A(p, c);
  if (tm.tl == 0) {
    tm.base[LU_INV] = inv;
    reinterpret_cast<int*>(&tm.base[LU_PIV])[0] = p;
  }
}
// elements of a rank-1 update that each lane of the first warp leaves to the other warps, in
// exchange for the look-ahead column it handles
#define LU_PANEL_SHARE 8
#endif

// In-place LU with partial pivoting of A (N x N): largest |a| in the column, lowest row on
// ties.  1/U_kk replaces U_kk on the diagonal, the composed row permutation (row i of P A is row
// perm[i] of A) goes to OFF_PERM, and the single-lane layout also keeps the pivot sequence.
__device__ void lu_factor(const Team& tm) {
#if TEAM == 1
  for (int k = 0; k < NEQ; ++k) {
    int p = k;
    long long best = abs_key(tm.A(k, k));
    for (int i = k + 1; i < NEQ; ++i) {
      const long long v = abs_key(tm.A(i, k));
      if (v > best) { best = v; p = i; }
    }
    tm.piv(k) = p;
    if (p != k)
      for (int j = 0; j < NEQ; ++j) { const double t = tm.A(k, j); tm.A(k, j) = tm.A(p, j); tm.A(p, j) = t; }
    const double inv = 1.0 / tm.A(k, k);
    tm.invd(k) = inv;
    for (int i = k + 1; i < NEQ; ++i) {
      const double l = tm.A(i, k) * inv;
      tm.A(i, k) = l;
      for (int j = k + 1; j < NEQ; ++j) tm.A(i, j) -= l * tm.A(k, j);
    }
  }
  for (int i = 0; i < NEQ; ++i) tm.perm(i) = i;
  for (int k = 0; k < NEQ; ++k) { const int p = tm.piv(k); if (p != k) { const int t = tm.perm(k); tm.perm(k) = tm.perm(p); tm.perm(p) = t; } }
#elif TEAM >= 128
  // Right-looking elimination with one column of look-ahead: while the team applies step k's
  // rank-1 update to columns k+2.., the first warp updates column k+1 and finds its pivot and the
  // pivot's inverse (lu_panel), so that the search, its reduction and the division stay off the
  // barrier-separated critical path: two barriers per column.  Every element receives the same
  // operations in the same order as in the column-by-column form.
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.perm(i) = i;
  if (tm.tl < 32) lu_panel(tm, 0);
  tsync();
  for (int k = 0; k < NEQ; ++k) {
    const int p = reinterpret_cast<const int*>(&tm.base[LU_PIV])[0];
    const double inv = tm.base[LU_INV];
    // rows k and p exchanged (every column but k), column k below the diagonal scaled by the
    // pivot's inverse, which replaces U_kk; the lane of row p also moves U_kk's old value
    if (p != k)
      for (int j = tm.tl; j < NEQ; j += TEAM)
        if (j != k) { const double t = tm.A(k, j); tm.A(k, j) = tm.A(p, j); tm.A(p, j) = t; }
    for (int i = k + 1 + tm.tl; i < NEQ; i += TEAM) {
      if (i == p) {
        const double t = tm.A(k, k);
        tm.A(k, k) = inv;
        tm.A(p, k) = t * inv;
      } else {
        tm.A(i, k) *= inv;
      }
    }
    if (tm.tl == 0) {
      if (p == k) {
        tm.A(k, k) = inv;
      } else {
        const int t = tm.perm(k);
        tm.perm(k) = tm.perm(p);
        tm.perm(p) = t;
      }
    }
    tsync();
    const int m = NEQ - k - 1;
    if (m > 0) {
      if (tm.tl < 32) lu_panel(tm, k + 1);
      // rank-1 update of rows k+1.., columns k+2.. (m x n2 elements in row-major order): the
      // first warp's lanes take the first e0 of them, LU_PANEL_SHARE fewer each than the others
      const int n2 = m - 1;
      if (n2 > 0) {
        const int tot = m * n2;
        int e0 = (tot - LU_PANEL_SHARE * (TEAM - 32)) * 32 / TEAM;
        e0 = e0 > 0 ? e0 : 0;
        int e, st, end;
        if (tm.tl < 32) { e = tm.tl; st = 32; end = e0; }
        else { e = e0 + tm.tl - 32; st = TEAM - 32; end = tot; }
        if (e < end) {
          int i = e / n2, j = e - (e / n2) * n2;
          const int qd = st / n2, rm = st - qd * n2;
          for (; e < end; e += st) {
            double& a = tm.A(k + 1 + i, k + 2 + j);
            a = fma(-tm.A(k + 1 + i, k), tm.A(k, k + 2 + j), a);
            i += qd;
            j += rm;
            if (j >= n2) { j -= n2; ++i; }
          }
        }
      }
      tsync();
    }
  }
#else
  // the composed permutation is built as the pivots are chosen (lane 0, after the row swap's
  // barrier), so no serial pass over the pivots is needed afterwards
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.perm(i) = i;
  for (int k = 0; k < NEQ; ++k) {
    // pivot search: (|a| key desc, row asc)
    long long best = -1;
    int p = NEQ;
    for (int i = k + tm.tl; i < NEQ; i += TEAM) {
      const long long v = abs_key(tm.A(i, k));
      if (v > best) { best = v; p = i; }
    }
    const unsigned msk = team_mask();
#pragma unroll
    for (int o = XOR0; o > 0; o >>= 1) {
      const long long vb = __shfl_xor_sync(msk, best, o);
      const int pb = __shfl_xor_sync(msk, p, o);
      if (vb > best || (vb == best && pb < p)) { best = vb; p = pb; }
    }
#if TEAM > 32
    {
      long long* rv = reinterpret_cast<long long*>(&tm.base[OFF_RED]);
      int* ri = reinterpret_cast<int*>(&tm.base[OFF_RED + 8]);
      if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = best; ri[threadIdx.x >> 5] = p; }
      __syncthreads();
      best = rv[0];
      p = ri[0];
      for (int w = 1; w < TEAM / 32; ++w)
        if (rv[w] > best || (rv[w] == best && ri[w] < p)) { best = rv[w]; p = ri[w]; }
      __syncthreads();
    }
#endif
    if (p != k)
      for (int j = tm.tl; j < NEQ; j += TEAM) { const double t = tm.A(k, j); tm.A(k, j) = tm.A(p, j); tm.A(p, j) = t; }
    tsync();
    // 1/pivot and the column scale by the first warp only: a warp-level FP64 instruction costs the
    // same pipe time whatever its lane count, so the other warps must not repeat the division
    if (tm.tl < 32) {
      const double inv = 1.0 / tm.A(k, k);
      __syncwarp(msk);  // every lane has read U_kk before lane 0 replaces it by its inverse
      if (tm.tl == 0) {
        tm.invd(k) = inv;
        if (p != k) { const int t = tm.perm(k); tm.perm(k) = tm.perm(p); tm.perm(p) = t; }
      }
      for (int i = k + 1 + tm.tl; i < NEQ; i += WL) tm.A(i, k) *= inv;
    }
    tsync();
    const int m = NEQ - k - 1;
    if (m > 0) {
      const int tot = m * m;
      const int qd = TEAM / m, rm = TEAM - qd * m;
      int i = tm.tl / m, j = tm.tl - (tm.tl / m) * m;
      for (int e = tm.tl; e < tot; e += TEAM) {
        tm.A(k + 1 + i, k + 1 + j) -= tm.A(k + 1 + i, k) * tm.A(k, k + 1 + j);
        i += qd;
        j += rm;
        if (j >= m) { j -= m; ++i; }
      }
    }
    tsync();
  }
#endif
}

#if TEAM >= 128 && NB >= 2 && NB <= TEAM / 32
// barrier of the solve's NB warps (barrier 0 is the team's)
__device__ __forceinline__ void solve_bar() {
  asm volatile("bar.sync 1, %0;" ::"r"(NB * 32) : "memory");
}
#endif

// Solve (LU) x = b in place on the vector at slot ob.  With TEAM > 1 only the first warp works,
// except for teams of four or more warps, where warp w holds rows 32w..32w+31.
__device__ void lu_solve(const Team& tm, int ob) {
#if TEAM == 1
  for (int k = 0; k < NEQ; ++k) {
    const int p = tm.piv(k);
    if (p != k) { const double t = tm.at(ob, k); tm.at(ob, k) = tm.at(ob, p); tm.at(ob, p) = t; }
  }
  for (int i = 0; i < NEQ; ++i) {
    double s = tm.at(ob, i);
    for (int j = 0; j < i; ++j) s -= tm.A(i, j) * tm.at(ob, j);
    tm.at(ob, i) = s;
  }
  for (int i = NEQ - 1; i >= 0; --i) {
    double s = tm.at(ob, i);
    for (int j = i + 1; j < NEQ; ++j) s -= tm.A(i, j) * tm.at(ob, j);
    tm.at(ob, i) = s * tm.invd(i);
  }
#elif TEAM >= 128 && NB >= 2 && NB <= TEAM / 32
  // Blocked substitution over NB warps, one 32-row block each, so that the FP64 work is spread
  // over the SM's sub-partitions instead of one: warp b solves its diagonal block (the finished
  // x_k broadcast by a shuffle, as below), publishes the block's values in the vector's slot, and
  // after a barrier of the NB warps the others apply the block's columns to their rows.  Every
  // row receives its updates in the same order (k increasing forward, decreasing backward) and
  // with the same operations as in the single-warp form.
  const int w = tm.tl >> 5, ln = tm.tl & 31;
  if (w < NB) {
    const int i = w * 32 + ln;
    double xr = i < NEQ ? tm.at(ob, tm.perm(i)) : 0.0;  // P b
    solve_bar();  // every entry of b is read before the slot receives x
    // L (unit lower) forward
    for (int b = 0; b < NB; ++b) {
      if (w == b) {
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
          const int k = b * 32 + kk;
          if (k < NEQ - 1) {
            const double xk = __shfl_sync(0xffffffffu, xr, kk);
            if (ln > kk && i < NEQ) xr = fma(-tm.A(i, k), xk, xr);
          }
        }
        if (i < NEQ) tm.at(ob, i) = xr;
      }
      if (b + 1 < NB) {
        solve_bar();
        if (w > b && i < NEQ) {
#pragma unroll 8
          for (int kk = 0; kk < 32; ++kk) {
            const int k = b * 32 + kk;
            xr = fma(-tm.A(i, k), tm.at(ob, k), xr);
          }
        }
      }
    }
    // U backward, 1/U_kk from the factorisation
    for (int b = NB - 1; b >= 0; --b) {
      if (w == b) {
#pragma unroll
        for (int kk = 31; kk >= 0; --kk) {
          const int k = b * 32 + kk;
          if (k < NEQ) {
            const double xk = __shfl_sync(0xffffffffu, xr, kk) * tm.invd(k);
            if (ln == kk) xr = xk;
            if (ln < kk) xr = fma(-tm.A(i, k), xk, xr);
          }
        }
        if (i < NEQ) tm.at(ob, i) = xr;
      }
      if (b > 0) {
        solve_bar();
        if (w < b) {
#pragma unroll 8
          for (int kk = 31; kk >= 0; --kk) {
            const int k = b * 32 + kk;
            if (k < NEQ) xr = fma(-tm.A(i, k), tm.at(ob, k), xr);
          }
        }
      }
    }
  }
  tsync();
#else
  // One warp, the vector in registers: lane l holds rows l, l + 32, ... (NB chunks).  Each
  // substitution step broadcasts the finished x_k with a shuffle and updates the rows it feeds,
  // so the dependent chain per step is a shuffle and an FMA, with no shared-memory round trip
  // and no barrier; the matrix loads do not depend on x and are issued ahead.  The update order
  // per row (k increasing forward, decreasing backward) is that of the column-oriented sweep.
  if (tm.tl < 32) {
    const int ln = tm.tl & (WL - 1);
    const unsigned msk = team_mask();
    double xr[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const int i = ln + WL * c;
      xr[c] = i < NEQ ? tm.at(ob, tm.perm(i)) : 0.0;  // P b
    }
    // L (unit lower) forward
#pragma unroll
    for (int kb = 0; kb < NB; ++kb) {
#pragma unroll
      for (int kk = 0; kk < WL; ++kk) {
        const int k = kb * WL + kk;
        if (k < NEQ - 1) {
          const double xk = __shfl_sync(msk, xr[kb], kk, WL);
#pragma unroll
          for (int c = kb; c < NB; ++c) {
            const int i = ln + WL * c;
            if ((c > kb || ln > kk) && i < NEQ) xr[c] = fma(-tm.A(i, k), xk, xr[c]);
          }
        }
      }
    }
    // U backward, 1/U_kk from the factorisation
#pragma unroll
    for (int kb = NB - 1; kb >= 0; --kb) {
#pragma unroll
      for (int kk = WL - 1; kk >= 0; --kk) {
        const int k = kb * WL + kk;
        if (k < NEQ) {
          const double xk = __shfl_sync(msk, xr[kb], kk, WL) * tm.invd(k);
          if (ln == kk) xr[kb] = xk;
#pragma unroll
          for (int c = 0; c <= kb; ++c) {
            const int i = ln + WL * c;
            if (c < kb || ln < kk) xr[c] = fma(-tm.A(i, k), xk, xr[c]);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const int i = ln + WL * c;
      if (i < NEQ) tm.at(ob, i) = xr[c];
    }
  }
  tsync();
#endif
}

#if TEAM > 1
// Column-oriented solve by the team's first warp through shared memory (the adjoint kernels use it: it needs
// no registers for the vector, and the adjoint kernels run at their register cap).
__device__ void lu_solve_col(const Team& tm, int ob) {
  if (tm.tl < 32) {
    const int ln = tm.tl & (WL - 1);
    const unsigned msk = team_mask();
    {  // P b through the composed permutation
      double g[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        const int i = ln + WL * c;
        g[c] = i < NEQ ? tm.at(ob, tm.perm(i)) : 0.0;
      }
      __syncwarp(msk);
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        const int i = ln + WL * c;
        if (i < NEQ) tm.at(ob, i) = g[c];
      }
    }
    __syncwarp(msk);
    for (int k = 0; k < NEQ - 1; ++k) {
      const double xk = tm.at(ob, k);
      for (int i = k + 1 + ln; i < NEQ; i += WL) tm.at(ob, i) -= tm.A(i, k) * xk;
      __syncwarp(msk);
    }
    for (int k = NEQ - 1; k >= 0; --k) {
      const double xk = tm.at(ob, k) * tm.invd(k);
      __syncwarp(msk);
      if (ln == (k & (WL - 1))) tm.at(ob, k) = xk;
      for (int i = ln; i < k; i += WL) tm.at(ob, i) -= tm.A(i, k) * xk;
      __syncwarp(msk);
    }
  }
  tsync();
}

#endif

// ------------------------------------------------------------------------------ ROS4 step

// One attempt of the s-stage Rosenbrock method of the generated header (Sec. 2.3, transformed
// form): coefficients rk_a, rk_c, rk_m, rk_e, gamma RGAM, RS stages; rk_newf[i] says whether stage
// i needs f at a new argument (1), reuses the previous stage's f (0: equal argument), or uses
// f(y) (2: the argument is y).  Size hh from y (OFF_Y): y_new into OFF_YT; returns the weighted
// RMS error (infinity if anything is non-finite).
// REG_SOLVE selects the register-resident stage solves, used for state vectors of more than 64
// entries (GB300, 111 species: +5% cells/s; at 53 species they measured 12% slower than the
// column-oriented sweep, at 13 species no different).  The adjoint's replay takes the column-oriented
// ones (same arithmetic in the same order) to stay within its register budget.
template <bool REG_SOLVE>
__device__ __forceinline__ void stage_solve(const Team& tm, int ob) {
#if TEAM > 1
  if (!REG_SOLVE) {
    lu_solve_col(tm, ob);
    return;
  }
#endif
  lu_solve(tm, ob);
}

template <bool REG_SOLVE = (NB >= 3)>
__device__ double ros4_attempt(const Team& tm, double P, double hh, double rtol, double atol,
                              const double* lnA_ext, double* rho = nullptr, double* wc = nullptr) {
#if ERK
  // explicit Runge-Kutta (RKF45) in increment form: u_i = hh f(y + sum_{j<i} a_ij u_j); no
  // Jacobian, no factorisation
#pragma unroll
  for (int st = 0; st < RS; ++st) {
    if (st > 0) {
      for (int i = tm.tl; i < NEQ; i += TEAM) {
        double v = tm.at(OFF_Y, i);
        for (int j = 0; j < st; ++j)
          if (rk_a[st * RS + j] != 0.0) v += rk_a[st * RS + j] * tm.at(UOFF(j), i);
        tm.at(OFF_YT, i) = v;
      }
      tsync();
    }
    eval_f(tm, st == 0 ? OFF_Y : OFF_YT, OFF_F, P, lnA_ext);
    const int ou = UOFF(st);
    for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(ou, i) = hh * tm.at(OFF_F, i);
    tsync();
  }
#else
  // stage 1: f0 into U1, M = I/(gamma h) - J (with a W-method cache: the cached factorisation
  // of I/(gamma h) - W when it was made for this step size and is young enough)
  const bool reuse = wc && wc[WC_H] == hh && wc[WC_AGE] < WAGE_MAX;
  if (reuse) {
    eval_f(tm, OFF_Y, OFF_U1, P, lnA_ext);
    for (int e = tm.tl; e < NEQ * NEQ; e += TEAM) tm.at(OFF_A, e) = wc[e];
    for (int e = tm.tl; e < PACKED_INTS(NEQ); e += TEAM) {
      tm.at(OFF_PERM, e) = wc[WC_PERM + e];
#if TEAM == 1
      tm.at(OFF_PIV, e) = wc[WC_PIV + e];
#endif
    }
    tsync();
  } else {
    eval_f_jac(tm, OFF_Y, OFF_U1, P, lnA_ext, -1.0, 1.0 / (RGAM * hh));
  }
  if (rho && !reuse) {
    // stiffness estimate: Gershgorin bound of the Jacobian scaled by the error weights,
    // max_i sum_j |J_ij| w_j / w_i with w = atol + rtol |y| (J_ij = -A_ij off the diagonal,
    // shift - A_ii on it)
    const double shift = 1.0 / (RGAM * hh);
    double mx = 0.0;
    for (int i = tm.tl; i < NEQ; i += TEAM) {
      double sum = 0.0;
      for (int j = 0; j < NEQ; ++j) {
        const double a = tm.A(i, j);
        sum += fabs(i == j ? shift - a : a) * (atol + rtol * fabs(tm.at(OFF_Y, j)));
      }
      const double r = sum / (atol + rtol * fabs(tm.at(OFF_Y, i)));
      mx = r > mx ? r : mx;
    }
    *rho = team_max(tm, mx);
  }
#if NEED_F0
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(OFF_F0, i) = tm.at(OFF_U1, i);
  tsync();
#endif
  if (!reuse) {
    lu_factor(tm);
    if (wc) {  // keep the factorisation for later attempts of this size
      for (int e = tm.tl; e < NEQ * NEQ; e += TEAM) wc[e] = tm.at(OFF_A, e);
      for (int e = tm.tl; e < PACKED_INTS(NEQ); e += TEAM) {
        wc[WC_PERM + e] = tm.at(OFF_PERM, e);
#if TEAM == 1
        wc[WC_PIV + e] = tm.at(OFF_PIV, e);
#endif
      }
      if (tm.tl == 0) { wc[WC_H] = hh; wc[WC_AGE] = 0.0; }
    }
  }
  stage_solve<REG_SOLVE>(tm, OFF_U1);
  const double ih = 1.0 / hh;
#pragma unroll
  for (int st = 1; st < RS; ++st) {
    if (rk_newf[st] == 1) {
      for (int i = tm.tl; i < NEQ; i += TEAM) {
        double v = tm.at(OFF_Y, i);
        for (int j = 0; j < st; ++j)
          if (rk_a[st * RS + j] != 0.0) v += rk_a[st * RS + j] * tm.at(UOFF(j), i);
        tm.at(OFF_YT, i) = v;
      }
      tsync();
      eval_f(tm, OFF_YT, OFF_F, P, lnA_ext);
    }
#if NEED_F0
    const int of = rk_newf[st] == 2 ? OFF_F0 : OFF_F;
#else
    const int of = OFF_F;
#endif
    const int ou = UOFF(st);
    for (int i = tm.tl; i < NEQ; i += TEAM) {
      double v = tm.at(of, i);
      for (int j = 0; j < st; ++j)
        if (rk_c[st * RS + j] != 0.0) v += (rk_c[st * RS + j] * ih) * tm.at(UOFF(j), i);
      tm.at(ou, i) = v;
    }
    tsync();
    stage_solve<REG_SOLVE>(tm, ou);
  }
#endif
  // new state, error estimate and its weighted RMS norm
  double acc = 0.0;
  bool bad = false;
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    const double y = tm.at(OFF_Y, i);
    double yn = y, e = 0.0;
#pragma unroll
    for (int j = 0; j < RS; ++j) {
      const double u = tm.at(UOFF(j), i);
      if (rk_m[j] != 0.0) yn += rk_m[j] * u;  // zero coefficients fold away at compile time
      if (rk_e[j] != 0.0) e += rk_e[j] * u;
    }
    tm.at(OFF_YT, i) = yn;
    const double ay = fabs(y), an = fabs(yn);
    const double sc = atol + rtol * (ay > an ? ay : an);
    const double z = e / sc;
    acc += z * z;
    if (!isfinite(yn)) bad = true;
  }
  acc = team_sum(tm, acc);
  bad = team_any(tm, bad);
  tsync();
  const double err = sqrt(acc / NEQ);
  return (bad || !isfinite(err)) ? __longlong_as_double(0x7ff0000000000000LL) : err;
}

// Controller state of one cell (team-uniform: every lane holds the same values).
struct Ctl {
  double t, h;
  int attempts, status;
  bool reject_last, done;
  bool acc;   // the last call accepted a step ...
  double hh;  // ... of this size
  bool want_rho;  // estimate the stiffness at the cell's first attempt (into rho)
  double rho;
  double* wc;     // the cell's W-method cache (global memory) or nullptr
};

// One attempt plus the controller decision (identical rules to the CPU oracle):
// fac = clamp(0.9 err^(-1/order), 0.2, 6) with err floored at 1e-10 (0.2 if non-finite); accept iff
// err <= 1; no growth right after a rejection; the last step is cut to land on dt (a step
// within 0.01% of the remainder is stretched to it); h_out is the controller's proposal after
// the last accepted step, or the proposal that the end cut shortened.
__device__ __forceinline__ void ros4_advance(const Team& tm, Ctl& c, double P, double dt, double rtol,
                                             double atol, int max_steps, double h_min,
                                             const double* lnA_ext) {
  c.acc = false;
  if (c.attempts >= max_steps) { c.status = ST_MAX_STEPS; c.done = true; return; }
  if (c.h < h_min) { c.status = ST_H_UNDERFLOW; c.done = true; return; }
  const bool last = c.t + 1.0001 * c.h >= dt;
  const double hh = last ? dt - c.t : c.h;
  const double err = ros4_attempt(tm, P, hh, rtol, atol, lnA_ext,
                                  (c.want_rho && c.attempts == 0) ? &c.rho : nullptr, c.wc);
  c.attempts++;
  const bool finite = isfinite(err);
  double fac = 0.2;
  if (finite) {
    const double e = err > 1e-10 ? err : 1e-10;
#if RORDER == 4
    fac = 0.9 / sqrt(sqrt(e));  // 0.9 err^(-1/order)
#elif RORDER == 3
    fac = 0.9 / cbrt(e);
#else
    fac = 0.9 * pow(e, -1.0 / RORDER);
#endif
    fac = fac < 0.2 ? 0.2 : (fac > 6.0 ? 6.0 : fac);
  }
  if (finite && err <= 1.0) {
    for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(OFF_Y, i) = tm.at(OFF_YT, i);
    if (c.wc && tm.tl == 0) c.wc[WC_AGE] += 1.0;  // the cached factorisation ages per accepted step
    tsync();
    if (c.reject_last && fac > 1.0) fac = 1.0;
    c.reject_last = false;
    c.acc = true;
    c.hh = hh;
    const double hnext = hh * fac;
    if (last) {
      c.h = hh < c.h ? c.h : hnext;
      c.done = true;
      c.status = ST_OK;
      return;
    }
    c.t += hh;
    c.h = hnext;
  } else {
    c.reject_last = true;
    c.h = hh * fac;
  }
}

// ------------------------------------------------------------------------------ cell I/O

__device__ __forceinline__ Team make_team(double* smem) {
  Team tm;
#if TEAM == 1
  tm.base = smem + threadIdx.x;
  tm.tl = 0;
#elif TEAM <= 32
  tm.base = smem + (threadIdx.x / TEAM) * TSTRIDE;
  tm.tl = threadIdx.x & (TEAM - 1);
#else
  tm.base = smem;
  tm.tl = threadIdx.x;
#endif
  return tm;
}

// y = [T, Y_k / W_k] into OFF_Y; returns false if any input is non-finite
__device__ __forceinline__ bool load_cell(const Team& tm, long long c, const double* T, const double* Y,
                                          long long ld) {
  bool bad = false;
  if (tm.tl == 0) {
    const double t = T[c];
    tm.at(OFF_Y, 0) = t;
    bad = !isfinite(t);
  }
  for (int k = tm.tl; k < NS - 1; k += TEAM) {
    const double v = Y[k * ld + c];
    tm.at(OFF_Y, 1 + k) = v * mk_invW[k];
    bad = bad || !isfinite(v);
  }
  bad = team_any(tm, bad);
  tsync();
  return !bad;
}

// T, Y back from OFF_Y; the bath-gas mass fraction from the closure
__device__ __forceinline__ void store_cell(const Team& tm, long long c, double* T, double* Y, long long ld) {
  double s = 0.0;
  for (int k = tm.tl; k < NS - 1; k += TEAM) {
    const double v = tm.at(OFF_Y, 1 + k) * mk_W[k];
    Y[k * ld + c] = v;
    s += v;
  }
  s = team_sum(tm, s);
  if (tm.tl == 0) {
    T[c] = tm.at(OFF_Y, 0);
    Y[(long long)(NS - 1) * ld + c] = 1.0 - s;
  }
}

// broadcast a team-lane-0 value
__device__ __forceinline__ long long team_bcast_ll(const Team& tm, long long v) {
#if TEAM == 1
  return v;
#elif TEAM <= 32
  return __shfl_sync(team_mask(), v, 0, TEAM);
#else
  long long* r = reinterpret_cast<long long*>(&tm.base[OFF_RED + 12]);
  if (tm.tl == 0) *r = v;
  __syncthreads();
  v = *r;
  __syncthreads();
  return v;
#endif
}

// ------------------------------------------------------------------------------ kernels

extern "C" __global__ void __launch_bounds__(TPB)
chem_eval_source_k(long long n_cells, const double* __restrict__ T, const double* __restrict__ P,
                   const double* __restrict__ n, double* __restrict__ f, long long ld,
                   const double* __restrict__ lnA_ext) {
  extern __shared__ double smem[];
  const Team tm = make_team(smem);
  const long long team_id = (long long)blockIdx.x * NTEAM + (TEAM <= 32 ? threadIdx.x / TEAM : 0);
  const long long stride = (long long)gridDim.x * NTEAM;
  for (long long c = team_id; c < n_cells; c += stride) {
    if (tm.tl == 0) tm.at(OFF_Y, 0) = T[c];
    for (int k = tm.tl; k < NS - 1; k += TEAM) tm.at(OFF_Y, 1 + k) = n[k * ld + c];
    tsync();
    eval_f(tm, OFF_Y, OFF_F, P[c], lnA_ext);
    for (int i = tm.tl; i < NEQ; i += TEAM) f[i * ld + c] = tm.at(OFF_F, i);
    tsync();
  }
}

extern "C" __global__ void __launch_bounds__(TPB)
chem_eval_jacobian_k(long long n_cells, const double* __restrict__ T, const double* __restrict__ P,
                     const double* __restrict__ n, double* __restrict__ J, long long ld,
                     const double* __restrict__ lnA_ext) {
  extern __shared__ double smem[];
  const Team tm = make_team(smem);
  const long long team_id = (long long)blockIdx.x * NTEAM + (TEAM <= 32 ? threadIdx.x / TEAM : 0);
  const long long stride = (long long)gridDim.x * NTEAM;
  for (long long c = team_id; c < n_cells; c += stride) {
    if (tm.tl == 0) tm.at(OFF_Y, 0) = T[c];
    for (int k = tm.tl; k < NS - 1; k += TEAM) tm.at(OFF_Y, 1 + k) = n[k * ld + c];
    tsync();
    eval_f_jac(tm, OFF_Y, OFF_U1, P[c], lnA_ext, 1.0, 0.0);  // f goes to U1: F aliases J scratch
    for (int e = tm.tl; e < NEQ * NEQ; e += TEAM) J[(long long)e * ld + c] = tm.at(OFF_A, e);
    tsync();
  }
}

// Per-cell method switching (chem_int_opts.cell_method): a launch of the alternative method's
// module (RKF45, or the W-method with its factorisation cache) runs the cells marked for it under
// their attempt budgets and keeps the input of any that fails; a launch of the Rosenbrock module
// runs the others and the failed ones and marks each cell for the next call:
//   * alternative RKF45 (AUTO_IMPLICIT): when dt * rho <= STIFF_BETA * attempts, rho the stiffness
//     estimate at the cell's first attempt (the explicit method's stability-limited steps, about
//     dt * rho / STIFF_BETA, would not outnumber the Rosenbrock attempts);
//   * alternative W-method (AUTO_IMPLICIT_W): when the cell took a single attempt and the
//     controller's next-step proposal is at least W_ENTRY_MARGIN * dt (a quiescent cell, whose
//     split steps the cached factorisation can serve; a cell whose one step only just fitted
//     would need many more steps of the second-order W-method); its cache is emptied, so the
//     W-method starts from a Jacobian at its own state;
// with budget 4 * attempts + 8; after a success of the alternative method with a attempts, it
// stays with budget 4a + 8.
#define AUTO_EXPLICIT 1
#define AUTO_IMPLICIT 2
#define AUTO_IMPLICIT_W 3
#define STIFF_BETA 3.0
#define W_ENTRY_MARGIN 2.0

// Persistent driver: each team pulls cells from the queue counter and integrates them to dt.
// With TEAM == 1 each thread refills independently (per-lane refill of retired cells); the
// loop body is one step attempt so that lanes on different cells still execute it together.
// Registers capped so that the cells that fit in shared memory can all be resident: eight
// 64-lane teams (53 species) or two 256-lane teams (111 species) per SM (GB300, 53 species
// at seven teams: 24.2K vs 22.7K cells/s with the cap)
// (sub-warp teams: 512 threads per SM, 128 registers a thread)
#define MIN_BLOCKS (TEAM == 64 ? 8 : (TEAM >= 128 ? 2 : (SUBWARP ? 512 / TPB : 1)))
extern "C" __global__ void __launch_bounds__(TPB, MIN_BLOCKS)
chem_integrate_k(long long n_cells, double* __restrict__ T, const double* __restrict__ P,
                 double* __restrict__ Y, long long ld, double dt, double rtol, double atol,
                 double* __restrict__ h_io, int* __restrict__ status_out,
                 int* __restrict__ attempts_out, const double* __restrict__ lnA_ext,
                 int max_steps, double h_min, double T_min, unsigned long long* queue,
                 int* __restrict__ tape_nacc, double* __restrict__ tape_h, double* __restrict__ tape_ck,
                 int tape_cap, int interval, const int* __restrict__ order,
                 const unsigned int* __restrict__ order_count, int keep_failed,
                 int* __restrict__ cell_method, int auto_mode, double* __restrict__ jac_cache) {
  extern __shared__ double smem[];
  const Team tm = make_team(smem);
  long long cell = -1;
  double Pc = 0.0;
  Ctl c;
  c.done = true;
  c.acc = false;
  c.want_rho = false;
  c.rho = 0.0;
  c.wc = nullptr;
  int nacc = 0;
  int ms_cell = max_steps;
  // queue positions: n_cells, or the device-held length of the cell list `order`
  const long long nq = order_count ? (long long)*order_count : n_cells;
  // bounded: every iteration either retires a cell or makes an attempt (<= max_steps per cell),
  // or consumes a queue position
  for (;;) {
    if (c.done) {
      long long nc = 0;
      if (tm.tl == 0) {
        const long long q = (long long)atomicAdd(queue, 1ULL);
        if (q >= nq) nc = n_cells;
        else if (order) nc = (order[q] >= 0 && order[q] < n_cells) ? order[q] : -1;
        else nc = q;
      }
      cell = team_bcast_ll(tm, nc);
      if (cell >= n_cells) break;
      if (cell < 0) continue;  // an invalid entry of the cell list: skipped
      Pc = P[cell];
      c.t = 0.0;
      c.h = h_io ? h_io[cell] : 0.0;
      if (!(c.h > 0.0)) c.h = dt;
      c.attempts = 0;
      c.status = ST_OK;
      c.reject_last = false;
      c.done = false;
      c.want_rho = auto_mode == AUTO_IMPLICIT;
      c.rho = 0.0;
      // the W-method's factorisation cache (not used by a Rosenbrock launch of the switching)
      c.wc = (jac_cache && auto_mode != AUTO_IMPLICIT_W) ? jac_cache + cell * (long long)WC_STRIDE : nullptr;
      // per-cell method switching: an explicit cell runs under its attempt budget
      ms_cell = max_steps;
      if (auto_mode == AUTO_EXPLICIT) {
        const int b = cell_method[cell];
        ms_cell = b > 0 && b < max_steps ? b : max_steps;
      }
      const bool ok = load_cell(tm, cell, T, Y, ld);
      nacc = 0;
      if (!ok || tm.at(OFF_Y, 0) < T_min) {
        if (tm.tl == 0) {
          if (status_out) status_out[cell] = ok ? ST_SKIPPED : ST_NONFINITE;
          if (attempts_out) attempts_out[cell] = 0;
          if (tape_nacc) tape_nacc[cell] = 0;
        }
        c.done = true;
        tsync();
        continue;
      }
      if (tape_ck)  // checkpoint 0: the initial state
        for (int i = tm.tl; i < NEQ; i += TEAM) tape_ck[(long long)i * n_cells + cell] = tm.at(OFF_Y, i);
    }
    if (tape_h && nacc >= tape_cap) {
      // the tape holds no further step: stop before attempting one, so that the stored state is
      // exactly the map the tape records (the adjoint then differentiates what was returned)
      c.status = ST_TAPE_FULL;
      c.done = true;
    } else {
      ros4_advance(tm, c, Pc, dt, rtol, atol, ms_cell, h_min, lnA_ext);
    }
    if (tape_h && c.acc && c.status != ST_TAPE_FULL) {
      // record the accepted step; checkpoint the state after every `interval` accepted steps
      if (tm.tl == 0) tape_h[(long long)nacc * n_cells + cell] = c.hh;
      ++nacc;
      if (nacc % interval == 0 && nacc < tape_cap)
        for (int i = tm.tl; i < NEQ; i += TEAM)
          tape_ck[((long long)(nacc / interval) * NEQ + i) * n_cells + cell] = tm.at(OFF_Y, i);
    }
    if (c.done) {
      if (tm.tl == 0 && tape_nacc) tape_nacc[cell] = nacc;
      // keep_failed: a cell that did not reach dt leaves its input state and step size in place
      // (a later launch integrates it again from the start)
      const bool keep = keep_failed && c.status != ST_OK;
      if (!keep) store_cell(tm, cell, T, Y, ld);
      if (tm.tl == 0) {
        if (h_io && !keep) h_io[cell] = c.h;
        if (status_out) status_out[cell] = c.status;
        if (attempts_out) attempts_out[cell] = c.attempts;
        if (auto_mode == AUTO_EXPLICIT)  // success: stay explicit, budget from this run
          cell_method[cell] = c.status == ST_OK ? 4 * c.attempts + 8 : 0;
        else if (auto_mode == AUTO_IMPLICIT)  // explicit next time if its stable steps are few
          cell_method[cell] = (c.status == ST_OK && dt * c.rho <= STIFF_BETA * c.attempts)
                                  ? 4 * c.attempts + 8 : 0;
        else if (auto_mode == AUTO_IMPLICIT_W) {  // the W-method next time if quiescent
          cell_method[cell] =
              (c.status == ST_OK && c.attempts == 1 && c.h >= W_ENTRY_MARGIN * dt) ? 12 : 0;
          if (jac_cache) jac_cache[cell * (long long)WC_STRIDE + WC_H] = 0.0;
        }
      }
      tsync();
    }
  }
}

// Cost-ordered work queue: a permutation of the cells by decreasing predicted cost (a counting
// sort over CHEM_ORDER_BINS cost buckets: histogram, descending exclusive scan, scatter).  Cells of
// equal cost are placed in no particular order.
#define ORDER_BINS 1024
extern "C" __global__ void chem_order_hist_k(long long n_cells, const int* __restrict__ cost,
                                             unsigned int* __restrict__ bins) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int v = cost[c];
  atomicAdd(&bins[v < 0 ? 0 : (v >= ORDER_BINS ? ORDER_BINS - 1 : v)], 1u);
}

// one block of ORDER_BINS threads: starts[b] = number of cells in bins above b
extern "C" __global__ void __launch_bounds__(ORDER_BINS) chem_order_scan_k(const unsigned int* __restrict__ bins,
                                                                          unsigned int* __restrict__ starts) {
  __shared__ unsigned int sh[ORDER_BINS];
  const int t = threadIdx.x;
  sh[t] = bins[ORDER_BINS - 1 - t];  // descending order of cost
  __syncthreads();
  for (int o = 1; o < ORDER_BINS; o <<= 1) {
    const unsigned int v = t >= o ? sh[t - o] : 0u;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  // inclusive scan over descending bins; exclusive start of bin b = inclusive value of its predecessor
  const int b = ORDER_BINS - 1 - t;
  starts[b] = t > 0 ? sh[t - 1] : 0u;
}

extern "C" __global__ void chem_order_scatter_k(long long n_cells, const int* __restrict__ cost,
                                                unsigned int* __restrict__ starts, int* __restrict__ order) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int v = cost[c];
  const unsigned int pos = atomicAdd(&starts[v < 0 ? 0 : (v >= ORDER_BINS ? ORDER_BINS - 1 : v)], 1u);
  order[pos] = (int)c;
}

// Per-cell method switching: split the cells into the explicit list (cell_method > 0) and the
// implicit list; counts[0], counts[1] their lengths (zeroed by the caller).
extern "C" __global__ void chem_route_k(long long n_cells, const int* __restrict__ cell_method,
                                        int* __restrict__ list_e, int* __restrict__ list_i,
                                        unsigned int* __restrict__ counts) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  if (cell_method[c] > 0) list_e[atomicAdd(&counts[0], 1u)] = (int)c;
  else list_i[atomicAdd(&counts[1], 1u)] = (int)c;
}

// After the explicit launch: its cells that ran out of budget (or step size) go to the end of the
// implicit list; the others' status is final and is copied to the caller's array.
extern "C" __global__ void chem_route_fallback_k(long long n_cells, const int* __restrict__ list_e,
                                                 unsigned int* __restrict__ counts, const int* __restrict__ st_e,
                                                 int* __restrict__ list_i, int* __restrict__ status_out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)counts[0]) return;
  const int c = list_e[q];
  if (c < 0 || c >= n_cells) return;
  const int s = st_e[c];
  if (s == ST_MAX_STEPS || s == ST_H_UNDERFLOW) list_i[atomicAdd(&counts[1], 1u)] = c;
  else if (status_out) status_out[c] = s;
}

// Plain driver, one launch per step attempt over all cells.  Per-cell controller state lives
// in the workspace: y [NEQ][n] (cell-fastest), t, h [n], packed flags/attempts/status [n].
struct PlainWs {
  double* y;
  double* t;
  double* h;
  int* flags;     // bit0 active, bit1 reject_last
  int* attempts;
  int* status;
  unsigned int* active_count;  // one counter per launch index
};

extern "C" __global__ void __launch_bounds__(TPB)
chem_plain_init_k(long long n_cells, const double* __restrict__ T, const double* __restrict__ Y,
                  long long ld, double dt, const double* __restrict__ h_in, double T_min,
                  double* wy, double* wt, double* wh, int* wflags, int* watt, int* wst) {
  extern __shared__ double smem[];
  const Team tm = make_team(smem);
  const long long team_id = (long long)blockIdx.x * NTEAM + (TEAM <= 32 ? threadIdx.x / TEAM : 0);
  const long long stride = (long long)gridDim.x * NTEAM;
  for (long long c = team_id; c < n_cells; c += stride) {
    const bool ok = load_cell(tm, c, T, Y, ld);
    for (int i = tm.tl; i < NEQ; i += TEAM) wy[i * n_cells + c] = tm.at(OFF_Y, i);
    if (tm.tl == 0) {
      double h = h_in ? h_in[c] : 0.0;
      if (!(h > 0.0)) h = dt;
      wt[c] = 0.0;
      wh[c] = h;
      watt[c] = 0;
      const bool skip = ok && tm.at(OFF_Y, 0) < T_min;
      wst[c] = ok ? (skip ? ST_SKIPPED : ST_OK) : ST_NONFINITE;
      wflags[c] = (ok && !skip) ? 1 : 0;
    }
    tsync();
  }
}

// same register cap as the persistent driver, so that the two differ only in how cells are scheduled
extern "C" __global__ void __launch_bounds__(TPB, MIN_BLOCKS)
chem_plain_attempt_k(long long n_cells, double* __restrict__ T, const double* __restrict__ P,
                     double* __restrict__ Y, long long ld, double dt, double rtol, double atol,
                     double* __restrict__ h_out, int* __restrict__ status_out,
                     int* __restrict__ attempts_out, const double* __restrict__ lnA_ext,
                     int max_steps, double h_min, double* wy, double* wt, double* wh, int* wflags,
                     int* watt, int* wst, unsigned int* active_count) {
  extern __shared__ double smem[];
  const Team tm = make_team(smem);
  const long long team_id = (long long)blockIdx.x * NTEAM + (TEAM <= 32 ? threadIdx.x / TEAM : 0);
  const long long stride = (long long)gridDim.x * NTEAM;
  for (long long cell = team_id; cell < n_cells; cell += stride) {
    const int fl = wflags[cell];
    if (!(fl & 1)) continue;  // team-uniform
    for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(OFF_Y, i) = wy[i * n_cells + cell];
    tsync();
    Ctl c;
    c.t = wt[cell];
    c.h = wh[cell];
    c.attempts = watt[cell];
    c.status = ST_OK;
    c.reject_last = (fl & 2) != 0;
    c.done = false;
    c.want_rho = false;
    c.wc = nullptr;
    ros4_advance(tm, c, P[cell], dt, rtol, atol, max_steps, h_min, lnA_ext);
    if (c.done) {
      store_cell(tm, cell, T, Y, ld);
      if (tm.tl == 0) {
        if (h_out) h_out[cell] = c.h;
        if (status_out) status_out[cell] = c.status;
        if (attempts_out) attempts_out[cell] = c.attempts;
        wflags[cell] = 0;
      }
    } else {
      for (int i = tm.tl; i < NEQ; i += TEAM) wy[i * n_cells + cell] = tm.at(OFF_Y, i);
      if (tm.tl == 0) {
        wt[cell] = c.t;
        wh[cell] = c.h;
        watt[cell] = c.attempts;
        wflags[cell] = 1 | (c.reject_last ? 2 : 0);
        atomicAdd(active_count, 1u);
      }
    }
    tsync();
  }
}

// Cells the plain driver never activated (non-finite or below T_min) get their status here.
extern "C" __global__ void chem_plain_finish_k(long long n_cells, int* __restrict__ status_out,
                                               int* __restrict__ attempts_out, const int* wst,
                                               const int* wflags_init_status) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const int s = wst[c];
  if (s == ST_SKIPPED || s == ST_NONFINITE) {
    if (status_out) status_out[c] = s;
    if (attempts_out) attempts_out[c] = 0;
  }
  (void)wflags_init_status;
}

// ============================================================================ discrete adjoint
// Gradients of a loss on the final state with respect to ln A of every reaction and to the
// initial state, through the ROS4 steps with the accepted step sizes frozen (Sec. 2.3 algebra,
// differentiated).  Only built for multi-lane teams (contiguous shared-memory layout), and only
// into the separately compiled adjoint module (CHEM_ADJOINT) so that forward modules compile fast.
#if TEAM >= 32 && defined(CHEM_ADJOINT) && TABLEAU_ID == 0

// forward-mode dual number: value and one directional derivative
struct DD {
  double v, d;
};
__device__ __forceinline__ DD mk(double v, double d) { DD r; r.v = v; r.d = d; return r; }
__device__ __forceinline__ DD operator+(DD a, DD b) { return mk(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ DD operator-(DD a, DD b) { return mk(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ DD operator-(DD a) { return mk(-a.v, -a.d); }
__device__ __forceinline__ DD operator*(DD a, DD b) { return mk(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ DD operator/(DD a, DD b) {
  const double q = a.v / b.v;
  return mk(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ DD operator+(DD a, double b) { return mk(a.v + b, a.d); }
__device__ __forceinline__ DD operator+(double b, DD a) { return mk(a.v + b, a.d); }
__device__ __forceinline__ DD operator-(DD a, double b) { return mk(a.v - b, a.d); }
__device__ __forceinline__ DD operator-(double b, DD a) { return mk(b - a.v, -a.d); }
__device__ __forceinline__ DD operator*(DD a, double b) { return mk(a.v * b, a.d * b); }
__device__ __forceinline__ DD operator*(double b, DD a) { return mk(a.v * b, a.d * b); }
__device__ __forceinline__ DD operator/(DD a, double b) { return mk(a.v / b, a.d / b); }
__device__ __forceinline__ DD operator/(double b, DD a) {
  const double q = b / a.v;
  return mk(q, -q * a.d / a.v);
}
__device__ __forceinline__ DD exp(DD a) { const double e = exp(a.v); return mk(e, e * a.d); }
__device__ __forceinline__ DD log(DD a) { return mk(log(a.v), a.d / a.v); }
__device__ __forceinline__ DD log10(DD a) { return mk(log10(a.v), a.d / (a.v * LN10)); }
__device__ __forceinline__ double vof(double a) { return a; }
__device__ __forceinline__ double vof(DD a) { return a.v; }
__device__ __forceinline__ double dof(double a) { return 0.0; }
__device__ __forceinline__ double dof(DD a) { return a.d; }
template <class S> struct S_is_dual { static constexpr bool value = false; };
template <> struct S_is_dual<DD> { static constexpr bool value = true; };
template <class S> __device__ __forceinline__ S szero();
template <> __device__ __forceinline__ double szero<double>() { return 0.0; }
template <> __device__ __forceinline__ DD szero<DD>() { return mk(0.0, 0.0); }
__device__ __forceinline__ void atomic_add_s(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_s(DD* p, DD v) {
  atomicAdd(&p->v, v.v);
  atomicAdd(&p->d, v.d);
}
__device__ __forceinline__ DD shfl_xor(DD a, int o) {
  return mk(__shfl_xor_sync(0xffffffffu, a.v, o), __shfl_xor_sync(0xffffffffu, a.d, o));
}
__device__ __forceinline__ double shfl_xor(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }

// adjoint slots, appended after the forward layout (units of doubles; DD arrays take 2 per entry)
#define AOFF_LAM SLOTS
#define AOFF_YB (AOFF_LAM + NEQ)
#define AOFF_UB (AOFF_YB + NEQ)
#define AOFF_W (AOFF_UB + 4 * NEQ)
#define AOFF_FB (AOFF_W + 4 * NEQ)
#define AOFF_Y2 (AOFF_FB + NEQ)
#define AOFF_Y3 (AOFF_Y2 + NEQ)
#define AOFF_V (AOFF_Y3 + NEQ)
#define AOFF_GP (AOFF_V + NEQ)
#define AOFF_TMP (AOFF_GP + NR)
#define AOFF_S (AOFF_TMP + NEQ)
// S-typed (2 doubles each) scratch of the VJP: state, gy, C, hRT, cp, ex, iex, dcp, atilde, Cbar,
// omega (11 x NS) and q (NR), plus 8 reduction slots
#define VS_Y 0
#define VS_GY (VS_Y + NEQ)
#define VS_C (VS_GY + NEQ)
#define VS_HRT (VS_C + NS)
#define VS_CP (VS_HRT + NS)
#define VS_EX (VS_CP + NS)
#define VS_IEX (VS_EX + NS)
#define VS_DCP (VS_IEX + NS)
#define VS_AT (VS_DCP + NS)
#define VS_CB (VS_AT + NS)
#define VS_OM (VS_CB + NS)
#define VS_Q (VS_OM + NS)
#define VS_RED (VS_Q + NR)
#define VS_TOTAL (VS_RED + 8 * TEAM / 32)
#define ASLOTS (AOFF_S + 2 * VS_TOTAL)

template <class S>
__device__ __forceinline__ S team_sum_s(const Team& tm, S v, S* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor(v, o);
#if TEAM > 32
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = red[0];
  for (int w = 1; w < TEAM / 32; ++w) v = v + red[w];
  __syncthreads();
#endif
  return v;
}

// Reverse-mode vector-Jacobian product of f at the state in VS_Y (type S):
//   gy = J(y)^T v  (into VS_GY)  and  gp_r += v^T d f / d lnA_r  (value part when S = double,
//   directional-derivative part when S = DD; accumulated into AOFF_GP).
// phi(y) = v^T f(y) = sum_k atilde_k omega_k with atilde_k = V v_{1+k} [k < bath]
// - v_T T V (h_k/RT) / cpm; gy = sum_k atilde_k d omega_k/dy + sum_k omega_k d atilde_k/dy.
template <class S>
__device__ void vjp(const Team& tm, double P, const double* __restrict__ lnA_ext) {
  S* sb = reinterpret_cast<S*>(&tm.base[AOFF_S]);
  S* Y = sb + VS_Y;
  const double* v = &tm.base[AOFF_V];
  double* gp = &tm.base[AOFF_GP];
  const S T = Y[0];
  const S invT = 1.0 / T;
  const S lnT = log(T);
  const S Z = szero<S>();
  S wsum = Z, nsum = Z;
  for (int k = tm.tl; k < NS - 1; k += TEAM) {
    wsum = wsum + mk_W[k] * Y[1 + k];
    nsum = nsum + Y[1 + k];
  }
  S* red = sb + VS_RED;
  wsum = team_sum_s(tm, wsum, red);
  nsum = team_sum_s(tm, nsum, red);
  const S nb = (1.0 - wsum) * mk_invW[BATH];
  const S V = (nsum + nb) * R_U * T / P;
  const S invV = 1.0 / V;
  S cpm = Z, dcpm = Z;
  for (int k = tm.tl; k < NS; k += TEAM) {
    const S n = k < NS - 1 ? Y[1 + k] : nb;
    sb[VS_C + k] = n * invV;
    const int r = vof(T) < mk_Tmid[k] ? 0 : 1;
    const double* c = mk_cp[k][r];
    const double* hh = mk_h[k][r];
    const double* s = mk_s[k][r];
    const double* d = mk_dcp[k][r];
    const S cp = c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
    const S hRT = hh[0] + T * (hh[1] + T * (hh[2] + T * (hh[3] + T * hh[4]))) + hh[5] * invT;
    const S sR = s[0] * lnT + s[6] + T * (s[1] + T * (s[2] + T * (s[3] + T * s[4])));
    const S dcp = d[0] + T * (d[1] + T * (d[2] + T * d[3]));
    const S ex = exp(sR - hRT);
    sb[VS_CP + k] = cp;
    sb[VS_HRT + k] = hRT;
    sb[VS_EX + k] = ex;
    sb[VS_IEX + k] = 1.0 / ex;
    sb[VS_DCP + k] = dcp;
    sb[VS_CB + k] = Z;
    cpm = cpm + n * cp;
    dcpm = dcpm + n * dcp;
  }
  cpm = team_sum_s(tm, cpm, red);
  dcpm = team_sum_s(tm, dcpm, red);
  const double vT = v[0];
  const S kT = vT * T * V / cpm;
  for (int k = tm.tl; k < NS; k += TEAM) {
    const S a0 = k < NS - 1 ? V * v[1 + k] : Z;
    sb[VS_AT + k] = a0 - kT * sb[VS_HRT + k];
  }
  tsync();
  const S Ctot = P * invT / R_U;
  const S rtp = R_U * T / P_ATM;
  const S irtp = 1.0 / rtp;
  S Tbar = Z, Bbar = Z;
  for (int r = tm.tl; r < NR; r += TEAM) {
    const int kind = mk_kind[r];
    const double lA = lnA_ext ? lnA_ext[mk_rorig[r]] : mk_lnA[r];
    const S kinf = exp(lA + mk_b[r] * lnT - mk_th[r] * invT);
    S kf = kinf;
    S dlkf_dT = (mk_b[r] + mk_th[r] * invT) * invT;
    S dlkf_dM = Z;
    S M = Z;
    S one_minus_g = Z + 1.0;  // d ln kf / d ln k_inf
    if (kind != ELEM) {
      M = Ctot;
      for (int e = mk_effoff[r]; e < mk_effoff[r + 1]; ++e) M = M + mk_effval[e] * sb[VS_C + mk_effsp[e]];
    }
    if (kind >= LIND) {
      const S k0 = exp(mk_lnA0[r] + mk_b0[r] * lnT - mk_th0[r] * invT);
      S Pr = k0 * M / kinf;
      bool floored = false;
      if (vof(Pr) < 1e-300) { Pr = Z + 1e-300; floored = true; }
      S F = Z + 1.0, dlF_dlPr = Z, dlF_dT = Z;
      if (kind == TROE) {
        const double a = mk_troe[r][0];
        const S e3 = exp(-T * mk_troe[r][1]);
        const S e1 = exp(-T * mk_troe[r][2]);
        const double T2 = mk_troe[r][3];
        const S e2 = T2 > 0.0 ? exp(-T2 * invT) : Z;
        const S Fc = (1.0 - a) * e3 + a * e1 + e2;
        const S lFc = log10(Fc);
        const S c = -0.4 - 0.67 * lFc;
        const S n = 0.75 - 1.27 * lFc;
        const S x = log10(Pr) + c;
        const S d = n - 0.14 * x;
        const S id = 1.0 / d;
        const S f1 = x * id;
        const S den = 1.0 / (1.0 + f1 * f1);
        const S lF = lFc * den;
        F = exp(lF * LN10);
        const S g2 = 2.0 * lFc * f1 * den * den;
        if (!floored) dlF_dlPr = -g2 * n * id * id;
        const S dFc = -(1.0 - a) * mk_troe[r][1] * e3 - a * mk_troe[r][2] * e1 +
                      (T2 > 0.0 ? T2 * invT * invT * e2 : Z);
        const S df1_dlFc = (-0.67 * n + 1.27 * x) * id * id;
        dlF_dT = (den - g2 * df1_dlFc) * dFc / Fc;
      }
      kf = kinf * (Pr / (1.0 + Pr)) * F;
      const S g = floored ? Z : 1.0 / (1.0 + Pr) + dlF_dlPr;
      const S dlk0 = (mk_b0[r] + mk_th0[r] * invT) * invT;
      dlkf_dM = g / M;
      dlkf_dT = dlkf_dT + g * (dlk0 - dlkf_dT) + dlF_dT;
      one_minus_g = 1.0 - g;
    }
    S kr = kf, fwd = kf, rev = Z + 1.0;
    const int nre = mk_nre[r], npr = mk_npr[r];
    S abar = Z;
    S dlKc = Z - mk_dnuf[r];
    for (int i = 0; i < nre; ++i) {
      const int sp = mk_rsp[r][i];
      for (int q = 0; q < mk_rnu[r][i]; ++q) { fwd = fwd * sb[VS_C + sp]; kr = kr * sb[VS_EX + sp]; }
      abar = abar - mk_rnuf[r][i] * sb[VS_AT + sp];
      dlKc = dlKc - mk_rnuf[r][i] * sb[VS_HRT + sp];
    }
    for (int i = 0; i < npr; ++i) {
      const int sp = mk_psp[r][i];
      for (int q = 0; q < mk_pnu[r][i]; ++q) { rev = rev * sb[VS_C + sp]; kr = kr * sb[VS_IEX + sp]; }
      abar = abar + mk_pnuf[r][i] * sb[VS_AT + sp];
      dlKc = dlKc + mk_pnuf[r][i] * sb[VS_HRT + sp];
    }
    const int dnu = mk_dnu[r];
    for (int q = 0; q < dnu; ++q) kr = kr * rtp;
    for (int q = 0; q < -dnu; ++q) kr = kr * irtp;
    rev = rev * kr;
    const S m = kind == THIRD ? M : Z + 1.0;
    const S qnet = fwd - rev;
    const S q = m * qnet;
    sb[VS_Q + r] = q;
    // parameter: d q / d lnA_r = q (d ln kf / d ln k_inf)
    const S gpr = abar * q * one_minus_g;
    gp[r] += S_is_dual<S>::value ? dof(gpr) : vof(gpr);
    dlKc = dlKc * invT;
    const S dqdT = m * (fwd * dlkf_dT - rev * (dlkf_dT - dlKc));
    Tbar = Tbar + abar * dqdT;
    if (kind != ELEM) {
      const S beta = kind == THIRD ? qnet : qnet * dlkf_dM;
      Bbar = Bbar + abar * beta;
      for (int e = mk_effoff[r]; e < mk_effoff[r + 1]; ++e)
        atomic_add_s(&sb[VS_CB + mk_effsp[e]], abar * beta * mk_effval[e]);
    }
    // d q / d C_j of the mass-action products
    for (int i = 0; i < nre; ++i) {
      const int nu = mk_rnu[r][i];
      S p = m * kf * mk_rnuf[r][i];
      for (int i2 = 0; i2 < nre; ++i2) {
        const int e = i2 == i ? nu - 1 : mk_rnu[r][i2];
        for (int t = 0; t < e; ++t) p = p * sb[VS_C + mk_rsp[r][i2]];
      }
      atomic_add_s(&sb[VS_CB + mk_rsp[r][i]], abar * p);
    }
    for (int i = 0; i < npr; ++i) {
      const int nu = mk_pnu[r][i];
      S p = -(m * kr * mk_pnuf[r][i]);
      for (int i2 = 0; i2 < npr; ++i2) {
        const int e = i2 == i ? nu - 1 : mk_pnu[r][i2];
        for (int t = 0; t < e; ++t) p = p * sb[VS_C + mk_psp[r][i2]];
      }
      atomic_add_s(&sb[VS_CB + mk_psp[r][i]], abar * p);
    }
  }
  Tbar = team_sum_s(tm, Tbar, red);
  Bbar = team_sum_s(tm, Bbar, red);
  tsync();
  // omega from q (fixed-order gather), and the mixture sums that use it
  S Q = Z, cpw = Z, vw = Z, Dbar = Z;
  for (int k = tm.tl; k < NS; k += TEAM) {
    S om = Z;
    for (int sg = mk_spseg_beg[k]; sg < mk_spseg_beg[k + 1]; ++sg)
      for (int e = mk_gseg_beg[sg]; e < mk_gseg_beg[sg + 1]; ++e) om = om + mk_gent_nu[e] * sb[VS_Q + mk_gent_rx[e]];
    sb[VS_OM + k] = om;
    Q = Q + sb[VS_HRT + k] * om;
    cpw = cpw + sb[VS_CP + k] * om;
    if (k < NS - 1) vw = vw + v[1 + k] * om;
    const S cb = sb[VS_CB + k] + Bbar;  // default third-body efficiency part on every C_j
    sb[VS_CB + k] = cb;
    Dbar = Dbar + cb * sb[VS_C + k];
  }
  Q = team_sum_s(tm, Q, red);
  cpw = team_sum_s(tm, cpw, red);
  vw = team_sum_s(tm, vw, red);
  Dbar = team_sum_s(tm, Dbar, red);
  tsync();
  const S Sp = vw - vT * T * Q / cpm;  // sum_k omega_k atilde_k / V
  const S RTP = R_U * T / P;
  const S icpm2 = 1.0 / (cpm * cpm);
  S* gy = sb + VS_GY;
  if (tm.tl == 0)
    gy[0] = Tbar - Dbar * invT + V * invT * Sp - vT * V * (cpw / cpm - T * Q * dcpm * icpm2);
  const S cbb = sb[VS_CB + BATH];
  const S cpb = sb[VS_CP + BATH];
  for (int j = tm.tl; j < NS - 1; j += TEAM) {
    const double w = mk_wratio[j];
    gy[1 + j] = (sb[VS_CB + j] - w * cbb) * invV - Dbar * RTP * (1.0 - w) * invV + RTP * (1.0 - w) * Sp +
                vT * T * V * Q * (sb[VS_CP + j] - w * cpb) * icpm2;
  }
  tsync();
}

// Solve M^T x = b in place at slot ob with the LU of P M (P M = L U, so M^T = U^T L^T P):
// U^T z = b forward, L^T t = z backward, x = P^T t.  The first warp works.
__device__ void lu_solve_T(const Team& tm, int ob) {
  if (tm.tl < 32) {
    const int ln = tm.tl;
    for (int i = ln; i < NEQ; i += 32) tm.at(AOFF_TMP, i) = tm.at(ob, i);
    __syncwarp();
    for (int i = 0; i < NEQ; ++i) {
      const double zi = tm.at(AOFF_TMP, i) * tm.invd(i);
      __syncwarp();
      if (ln == (i & 31)) tm.at(AOFF_TMP, i) = zi;
      for (int k = i + 1 + ln; k < NEQ; k += 32) tm.at(AOFF_TMP, k) -= tm.A(i, k) * zi;
      __syncwarp();
    }
    for (int i = NEQ - 1; i > 0; --i) {
      const double ti = tm.at(AOFF_TMP, i);
      for (int k = ln; k < i; k += 32) tm.at(AOFF_TMP, k) -= tm.A(i, k) * ti;
      __syncwarp();
    }
    for (int i = ln; i < NEQ; i += 32) tm.at(ob, tm.perm(i)) = tm.at(AOFF_TMP, i);
  }
  tsync();
}

// VJP at the state in slot oy (double) with weights at AOFF_V; gy added to yb scaled by the
// coefficients of up to three destinations: dst[0] += c0 gy, ...
template <class S>
__device__ __forceinline__ void set_vjp_state(const Team& tm, int oy, int odir) {
  S* sb = reinterpret_cast<S*>(&tm.base[AOFF_S]);
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    S v;
    if constexpr (S_is_dual<S>::value) v = mk(tm.at(oy, i), tm.at(odir, i));
    else v = tm.at(oy, i);
    sb[VS_Y + i] = v;
  }
  tsync();
}

__device__ __forceinline__ void add_gy(const Team& tm, bool dual, int o1, double c1, int o2, double c2, int o3, double c3) {
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    double g;
    if (dual) g = reinterpret_cast<const DD*>(&tm.base[AOFF_S])[VS_GY + i].d;
    else g = reinterpret_cast<const double*>(&tm.base[AOFF_S])[VS_GY + i];
    if (o1 >= 0) tm.at(o1, i) += c1 * g;
    if (o2 >= 0) tm.at(o2, i) += c2 * g;
    if (o3 >= 0) tm.at(o3, i) += c3 * g;
  }
  tsync();
}

// Adjoint of one frozen-h ROS4 step y_n -> y_{n+1}: on entry OFF_Y = y_n and AOFF_LAM =
// dL/dy_{n+1}; on exit AOFF_LAM = dL/dy_n, and dL/dlnA accumulated in AOFF_GP.
// Forward: M = I/(gamma h) - J(y), u_i = M^-1 r_i, r_1 = f(y), r_2 = f(Y2) + c21/h u1,
// r_3 = f(Y3) + (c31 u1 + c32 u2)/h, r_4 = f(Y3) + (c41 u1 + c42 u2 + c43 u3)/h,
// Y2 = y + a21 u1, Y3 = y + a31 u1 + a32 u2, y_{n+1} = y + sum m_i u_i.
// Reverse: ubar_i = m_i lambda, w_i = M^-T ubar_i (taken in the order 4, 3, 2, 1 as each ubar_i
// becomes final), fbar pulls back through J(Y)^T and d f / d lnA (VJP), and M's dependence on
// J(y) adds sum_i d/dy [w_i^T J(y) u_i] and d/dlnA [w_i^T J(y) u_i] (dual-number VJPs at y along
// u_i with weights w_i).
__device__ void adjoint_step(const Team& tm, double P, double h, const double* lnA_ext) {
  const int U1 = OFF_U1, U2 = OFF_U2, U3 = OFF_U3, U4 = OFF_U4;
  const int W1 = AOFF_W, W2 = AOFF_W + NEQ, W3 = AOFF_W + 2 * NEQ, W4 = AOFF_W + 3 * NEQ;
  const int B1 = AOFF_UB, B2 = AOFF_UB + NEQ, B3 = AOFF_UB + 2 * NEQ, B4 = AOFF_UB + 3 * NEQ;
  const double ih = 1.0 / h;
  // ---- forward recompute
  eval_f_jac(tm, OFF_Y, U1, P, lnA_ext, -1.0, 1.0 / (RGAM * h));
  lu_factor(tm);
  lu_solve_col(tm, U1);
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    const double v = tm.at(OFF_Y, i) + RA21 * tm.at(U1, i);
    tm.at(OFF_YT, i) = v;
    tm.at(AOFF_Y2, i) = v;
  }
  tsync();
  eval_f(tm, OFF_YT, OFF_F, P, lnA_ext);
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(U2, i) = tm.at(OFF_F, i) + (RC21 * ih) * tm.at(U1, i);
  tsync();
  lu_solve_col(tm, U2);
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    const double v = tm.at(OFF_Y, i) + RA31 * tm.at(U1, i) + RA32 * tm.at(U2, i);
    tm.at(OFF_YT, i) = v;
    tm.at(AOFF_Y3, i) = v;
  }
  tsync();
  eval_f(tm, OFF_YT, OFF_F, P, lnA_ext);
  for (int i = tm.tl; i < NEQ; i += TEAM)
    tm.at(U3, i) = tm.at(OFF_F, i) + (RC31 * ih) * tm.at(U1, i) + (RC32 * ih) * tm.at(U2, i);
  tsync();
  lu_solve_col(tm, U3);
  for (int i = tm.tl; i < NEQ; i += TEAM)
    tm.at(U4, i) = tm.at(OFF_F, i) + (RC41 * ih) * tm.at(U1, i) + (RC42 * ih) * tm.at(U2, i) +
                   (RC43 * ih) * tm.at(U3, i);
  tsync();
  lu_solve_col(tm, U4);
  // ---- reverse
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    const double l = tm.at(AOFF_LAM, i);
    tm.at(AOFF_YB, i) = l;
    tm.at(B1, i) = RM1 * l;
    tm.at(B2, i) = RM2 * l;
    tm.at(B3, i) = RM3 * l;
    tm.at(B4, i) = RM4 * l;
  }
  tsync();
  // stage 4
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(W4, i) = tm.at(B4, i);
  tsync();
  lu_solve_T(tm, W4);
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    const double w = tm.at(W4, i);
    tm.at(AOFF_FB, i) = w;
    tm.at(B1, i) += (RC41 * ih) * w;
    tm.at(B2, i) += (RC42 * ih) * w;
    tm.at(B3, i) += (RC43 * ih) * w;
  }
  tsync();
  // stage 3
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(W3, i) = tm.at(B3, i);
  tsync();
  lu_solve_T(tm, W3);
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    const double w = tm.at(W3, i);
    tm.at(AOFF_FB, i) += w;
    tm.at(AOFF_V, i) = tm.at(AOFF_FB, i);
    tm.at(B1, i) += (RC31 * ih) * w;
    tm.at(B2, i) += (RC32 * ih) * w;
  }
  tsync();
  set_vjp_state<double>(tm, AOFF_Y3, AOFF_Y3);
  vjp<double>(tm, P, lnA_ext);
  add_gy(tm, false, AOFF_YB, 1.0, B1, RA31, B2, RA32);
  // stage 2
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(W2, i) = tm.at(B2, i);
  tsync();
  lu_solve_T(tm, W2);
  for (int i = tm.tl; i < NEQ; i += TEAM) {
    const double w = tm.at(W2, i);
    tm.at(AOFF_V, i) = w;
    tm.at(B1, i) += (RC21 * ih) * w;
  }
  tsync();
  set_vjp_state<double>(tm, AOFF_Y2, AOFF_Y2);
  vjp<double>(tm, P, lnA_ext);
  add_gy(tm, false, AOFF_YB, 1.0, B1, RA21, -1, 0.0);
  // stage 1
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(W1, i) = tm.at(B1, i);
  tsync();
  lu_solve_T(tm, W1);
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(AOFF_V, i) = tm.at(W1, i);
  tsync();
  set_vjp_state<double>(tm, OFF_Y, OFF_Y);
  vjp<double>(tm, P, lnA_ext);
  add_gy(tm, false, AOFF_YB, 1.0, -1, 0.0, -1, 0.0);
  // M = I/(gamma h) - J(y): second-order terms along each u_i with weights w_i
  for (int st = 0; st < 4; ++st) {
    for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(AOFF_V, i) = tm.at(AOFF_W + st * NEQ, i);
    tsync();
    set_vjp_state<DD>(tm, OFF_Y, UOFF(st));
    vjp<DD>(tm, P, lnA_ext);
    add_gy(tm, true, AOFF_YB, 1.0, -1, 0.0, -1, 0.0);
  }
  for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(AOFF_LAM, i) = tm.at(AOFF_YB, i);
  tsync();
}

// Scratch of chem_adjoint_noalloc (the adjoint for callers that cannot allocate device memory):
// a fixed array in this module, CHEM_ADJ_SCRATCH_BYTES long, shared by every call on this
// module; the host resolves its device address once per loaded module.
static __device__ __align__(256) double chem_adj_scratch[CHEM_ADJ_SCRATCH_BYTES / 8];

__device__ __forceinline__ long long team_global_id() {
  return (long long)blockIdx.x * NTEAM + (TEAM == 32 ? (threadIdx.x >> 5) : 0);
}

// Reverse sweep over every cell's checkpointed forward: per cell, segments of `interval`
// accepted steps are recomputed from their checkpoint (states kept in this team's slice of
// `seg`), then stepped through backwards.  dL/dlnA is accumulated per team and written to
// gp_partial[team][r]; chem_adjoint_reduce_k sums the teams in a fixed order.
// (one block per SM as the register bound: the adjoint's shared memory already limits residency
// to four 64-lane or one 256-lane team per SM, so the registers go to avoiding spills)
extern "C" __global__ void __launch_bounds__(TPB, 1)
chem_adjoint_k(long long n_cells, const double* __restrict__ P, const double* __restrict__ gT,
               const double* __restrict__ gY, long long ld, double* __restrict__ gT0,
               double* __restrict__ gY0, const double* __restrict__ lnA_ext,
               const int* __restrict__ tape_nacc, const double* __restrict__ tape_h,
               const double* __restrict__ tape_ck, int interval, double* __restrict__ seg,
               double* __restrict__ gp_partial, unsigned long long* queue) {
  extern __shared__ double smem[];
  const Team tm = make_team(smem);
  const long long tg = team_global_id();
  for (int r = tm.tl; r < NR; r += TEAM) tm.at(AOFF_GP, r) = 0.0;
  tsync();
  double* segc = seg + tg * (long long)interval * NEQ;
  for (;;) {
    long long nc = 0;
    if (tm.tl == 0) nc = (long long)atomicAdd(queue, 1ULL);
    const long long cell = team_bcast_ll(tm, nc);
    if (cell >= n_cells) break;
    const int nacc = tape_nacc[cell];
    const double Pc = P[cell];
    const double gb = gY[(long long)BATH * ld + cell];
    if (tm.tl == 0) tm.at(AOFF_LAM, 0) = gT[cell];
    for (int k = tm.tl; k < NS - 1; k += TEAM) tm.at(AOFF_LAM, 1 + k) = mk_W[k] * (gY[k * ld + cell] - gb);
    tsync();
    for (int sg = (nacc - 1) / interval; nacc > 0 && sg >= 0; --sg) {
      const int s0 = sg * interval;
      const int s1 = min(nacc, s0 + interval);
      for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(OFF_Y, i) = tape_ck[((long long)sg * NEQ + i) * n_cells + cell];
      tsync();
      for (int s = s0; s < s1; ++s) {
        for (int i = tm.tl; i < NEQ; i += TEAM) segc[(s - s0) * NEQ + i] = tm.at(OFF_Y, i);
        if (s + 1 < s1) {
          ros4_attempt<false>(tm, Pc, tape_h[(long long)s * n_cells + cell], 1.0, 1.0, lnA_ext);
          for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(OFF_Y, i) = tm.at(OFF_YT, i);
        }
        tsync();
      }
      for (int s = s1 - 1; s >= s0; --s) {
        for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(OFF_Y, i) = segc[(s - s0) * NEQ + i];
        tsync();
        adjoint_step(tm, Pc, tape_h[(long long)s * n_cells + cell], lnA_ext);
      }
    }
    // initial state y0 = [T0, Y0_k / W_k]; the bath mass fraction does not enter y0
    if (tm.tl == 0) {
      gT0[cell] = tm.at(AOFF_LAM, 0);
      gY0[(long long)BATH * ld + cell] = 0.0;
    }
    for (int k = tm.tl; k < NS - 1; k += TEAM) gY0[k * ld + cell] = tm.at(AOFF_LAM, 1 + k) * mk_invW[k];
    tsync();
  }
  for (int r = tm.tl; r < NR; r += TEAM) gp_partial[tg * NR + r] = tm.at(AOFF_GP, r);
}

extern "C" __global__ void chem_adjoint_reduce_k(long long n_parts, const double* __restrict__ gp_partial,
                                                 double* __restrict__ g_lnA) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= NR) return;
  double s = 0.0;
  for (long long t = 0; t < n_parts; ++t) s += gp_partial[t * NR + r];
  g_lnA[mk_rorig[r]] = s;  // mechanism order
}

// Vector-Jacobian products per cell (parity entry point of the adjoint's building block):
// gy = J(y)^T v  [NEQ x ld], gp = (d f / d lnA)^T v  [NR x ld].
extern "C" __global__ void __launch_bounds__(TPB)
chem_eval_vjp_k(long long n_cells, const double* __restrict__ T, const double* __restrict__ P,
                const double* __restrict__ n, const double* __restrict__ v, double* __restrict__ gy,
                double* __restrict__ gp, long long ld, const double* __restrict__ lnA_ext) {
  extern __shared__ double smem[];
  const Team tm = make_team(smem);
  const long long stride = (long long)gridDim.x * NTEAM;
  for (long long c = team_global_id(); c < n_cells; c += stride) {
    if (tm.tl == 0) tm.at(OFF_Y, 0) = T[c];
    for (int k = tm.tl; k < NS - 1; k += TEAM) tm.at(OFF_Y, 1 + k) = n[k * ld + c];
    for (int i = tm.tl; i < NEQ; i += TEAM) tm.at(AOFF_V, i) = v[i * ld + c];
    for (int r = tm.tl; r < NR; r += TEAM) tm.at(AOFF_GP, r) = 0.0;
    tsync();
    set_vjp_state<double>(tm, OFF_Y, OFF_Y);
    vjp<double>(tm, P[c], lnA_ext);
    const double* g = reinterpret_cast<const double*>(&tm.base[AOFF_S]) + VS_GY;
    for (int i = tm.tl; i < NEQ; i += TEAM) gy[i * ld + c] = g[i];
    for (int r = tm.tl; r < NR; r += TEAM) gp[(long long)mk_rorig[r] * ld + c] = tm.at(AOFF_GP, r);
    tsync();
  }
}

#endif  // TEAM >= 32 && CHEM_ADJOINT

extern "C" __device__ const int chem_aslots =
#if TEAM >= 32 && defined(CHEM_ADJOINT) && TABLEAU_ID == 0
    ASLOTS;
#else
    0;
#endif
