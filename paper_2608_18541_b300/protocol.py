"""Switching statistics of the paper's GdFeCo protocol (Sec. II.G): a run
switches when the Gd sublattice z-magnetisation has reversed sign and stays
reversed from the end of the cooling stage to the end of the run;
probabilities over independent realisations carry Wilson 95 % intervals.
Host-side analysis of the observable rows (no device work)."""
import math

# columns of an observable row
COL_T = 0
COL_MZ_GD = 6          # species 1 (Gd), z component


def gd_switched(rows, t_cool_end, initial_sign=-1.0):
    """rows: observable rows of one realisation (time-ordered).  True when
    every row at or after t_cool_end has m_z(Gd) of the sign opposite to the
    initial one (and there is at least one such row)."""
    late = [r for r in rows if r[COL_T] >= t_cool_end * (1 - 1e-12)]
    return bool(late) and all(r[COL_MZ_GD] * initial_sign < 0.0 for r in late)


def wilson_interval(k, n, z=1.959963984540054):
    """Wilson score interval of a binomial proportion k/n."""
    if n <= 0:
        raise ValueError("n must be positive")
    p = k / n
    den = 1.0 + z * z / n
    centre = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return max(0.0, centre - half), min(1.0, centre + half)
