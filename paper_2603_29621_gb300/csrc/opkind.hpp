// Operator kinds and stabilised-NS term flags (host and device).
#pragma once

namespace mfns {

// OP_VMASS: the velocity mass (u, v) of the Stokes space's velocity block, Dirichlet velocity entries
// held at zero (the M of the space-time operator, Section 4).
enum OpKind : int { OP_STOKES_A = 0, OP_STOKES = 1, OP_STAB_NS = 2, OP_PMASS = 3, OP_VMASS = 4 };
enum Terms : int {
  TERM_MASS = 1, TERM_CONV = 2, TERM_NEWTON = 4, TERM_SUPG = 8,
  TERM_SUPG_NEWTON = 16, TERM_PSPG = 32, TERM_STRONG_VISC = 64
};

}  // namespace mfns
