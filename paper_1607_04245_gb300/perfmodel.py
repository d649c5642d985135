"""The paper's thread-transposition sizes and its traffic/flop model (Sec. 3, Sec. 3.3).

Used for reporting only: the benchmark quotes a "paper-model GF/s" next to its own
flop count, because the paper's GF/s figures are computed with this model. The
kernels of this library do not use thread transposition; these formulas describe
the paper's design, not ours.
"""

from __future__ import annotations

import dataclasses
import math


@dataclasses.dataclass(frozen=True)
class TransposeSizes:
    """Sizes of one cell batch of the paper's kernel (Sec. 3, Figs. 1-3)."""

    N_b: int  # scalar basis functions per cell
    N_q: int  # quadrature points per cell
    N_comp: int = 1  # field components
    N_bl: int = 1  # concurrent cell blocks per batch

    @property
    def N_bt(self) -> int:  # total basis functions over all components
        return self.N_b * self.N_comp

    @property
    def N_bs(self) -> int:  # cells in one block: LCM(N_b, N_q)
        return math.lcm(self.N_b, self.N_q)

    @property
    def N_bc(self) -> int:  # cells per batch
        return self.N_bs * self.N_bl

    @property
    def N_t(self) -> int:  # threads per thread block
        return self.N_bc * self.N_comp

    @property
    def N_sqc(self) -> int:  # cells each thread handles in the quadrature phase
        return self.N_bs // self.N_b

    @property
    def N_sbc(self) -> int:  # cells each thread handles in the basis phase
        return self.N_bs // self.N_q

    @property
    def N_tq(self) -> int:  # threads per cell in the quadrature phase
        return self.N_q * self.N_comp


def batch_flops(d: int, s: TransposeSizes) -> int:
    """Flops per cell batch (Sec. 3.3):
    [((2 + (2 + 2d) d) N_bt + 2 d N_comp) N_q + (2 + 2d) d N_q N_bt] N_bs N_bl."""
    per_block = ((2 + (2 + 2 * d) * d) * s.N_bt + 2 * d * s.N_comp) * s.N_q + (2 + 2 * d) * d * s.N_q * s.N_bt
    return per_block * s.N_bs * s.N_bl


def batch_bytes(d: int, s: TransposeSizes, word: int = 4) -> int:
    """Bytes loaded per cell batch (Sec. 3.3): word * N_t ((d^2 + 1) + N_bt + (d + 1) N_q).
    The paper writes it for 4-byte words; ``word`` = 8 gives the double-precision count."""
    return word * s.N_t * ((d * d + 1) + s.N_bt + (d + 1) * s.N_q)


def beta(d: int, s: TransposeSizes):
    """Algorithmic balance in flop/byte, as an exact fraction (numerator, denominator)."""
    f, b = batch_flops(d, s), batch_bytes(d, s)
    g = math.gcd(f, b)
    return f // g, b // g


def flops_per_cell(d: int, N_q: int, N_comp: int) -> float:
    """Paper-model flops per cell for a P1 simplex (N_b = d + 1)."""
    s = TransposeSizes(N_b=d + 1, N_q=N_q, N_comp=N_comp)
    return batch_flops(d, s) / s.N_bc


def shared_bytes(d: int, s: TransposeSizes, word: int = 4) -> int:
    """Upper bound on shared memory per thread block (Sec. 3.3):
    M = word ((d^2 + 1) N_t + (d + 1) N_bt N_q + N_t N_bt + (d + 1) N_t N_sqc)."""
    return word * ((d * d + 1) * s.N_t + (d + 1) * s.N_bt * s.N_q + s.N_t * s.N_bt + (d + 1) * s.N_t * s.N_sqc)


def collapsed_laplacian_flops(d: int, N_q: int) -> int:
    """Floating-point operations per cell of this library's collapsed P1 Laplacian (an FMA
    counts as 2), i.e. the arithmetic of r_b = (Kbar / |det J|) n_b . h that the kernels
    execute in place of the per-point loops of the paper's model:
      Jacobian columns x_j - x_0                      d^2 subtractions
      adjugate rows n_j (2x2: negations; 3x3: cross products of two columns each)
                                                      d = 3: 9 (mul + fma) = 27; d = 2: 0
      det J = e_0 . n_0 (3D) or a 2x2 determinant     2d - 1
      Kbar = sum_q w_q K_q                            2 N_q - 1
      s = Kbar / |det J|                              1
      du_j = u_j - u_0                                d
      h = sum_j du_j n_j                              d (2d - 1)
      n_j . h for j = 1..d                            d (2d - 1)
      r_j = s (n_j . h)                               d
      r_0 = -(r_1 + ... + r_d)                        d - 1
    The compensated sum and the float64 fallback of the mixed form are not counted."""
    adj = 27 if d == 3 else 0
    det = 2 * d - 1 if d == 3 else 3
    return d * d + adj + det + (2 * N_q - 1) + 1 + d + 2 * d * (2 * d - 1) + d + (d - 1)
