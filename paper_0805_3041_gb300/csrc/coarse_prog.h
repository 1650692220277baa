// coarse_prog.h -- step codes of the single-CTA coarse-cycle program (kernels_coarse.cu).
// A program is an array of int4 {code, level, a, b}; the CTA runs the steps in order
// with a barrier after each.
#pragma once

namespace mg {

enum CoarseOp {
  CP_LOAD_G = 1,    // g_y <- global g (padded layout of level y)
  CP_LOAD_U = 2,    // u_y[a] <- global u
  CP_STORE_U = 3,   // global u <- u_y[a] (unknowns)
  CP_ZERO_U = 4,    // u_y[a] = 0
  CP_JACOBI = 5,    // u_y[b] = u_y[a] + omega D^-1 (g - A u_y[a]);  a < 0: from a zero iterate
  CP_RB_HALF = 6,   // red-black half sweeps on u_y[b], in place: a = first colour | zero << 1 |
                    // (count - 1) << 2, colours alternating, one barrier between them; zero: the
                    // first half sweep starts from a zero iterate and sets every unknown
  CP_LINE = 7,      // a = dir | zebra << 1 | colour << 2,  b = src | dst << 4 | scratch << 8;
                    // r, scratch and the level's z array hold the elimination
  CP_DEFECT = 8,    // r_y = g_y - A u_y[a]; b = 1: then g_{y-1} = R r_y in the same step
  CP_RESTRICT = 9,  // g_{y-1} = R r_y  (a = 1: R g_y, the right-hand side itself)
  CP_PROLONG = 10,  // u_y[a] += omega_l P u_{y-1}[b & 1]; b >> 1 = d + 1: then the red-black sweeps
                    // of descriptor d (as CP_RB_HALF) on u_y[a] in the same step
  CP_COARSE = 11,   // u_1[a] = A_1^{-1} g_1
  CP_INTERP = 13,   // u_y[a] = P u_{y-1}[b]  (interpolation of a coarse solution, weight 1)
  CP_ADAPT = 14     // u_y[a] += omega P e, e = u_{y-1}[b], omega = (g_y - A u_y[a], P e) / (A P e, P e)
                    // (the energy-optimal correction weight; r_y holds P e afterwards)
};

}  // namespace mg
