"""Three-temperature relaxation analysis (paper Sec. III): T_e, the ion
(lattice) temperature and the spin temperature from the observable rows of a
moving-lattice run, and the lattice equilibration time -- the first time the
lattice temperature covers 90 % of its range.  Host-side analysis."""
import numpy as np

COL_T, COL_TSPIN0, COL_TE, COL_TL = 0, 13, 15, 16


def t90(t, T, tail=0.1):
    """First time at which T has covered 90 % of the way from T[0] to its
    final value (the mean over the last `tail` fraction of the samples)."""
    t = np.asarray(t, dtype=float)
    T = np.asarray(T, dtype=float)
    k = max(1, int(round(tail * T.size)))
    Tf = T[-k:].mean()
    target = T[0] + 0.9 * (Tf - T[0])
    sgn = 1.0 if Tf >= T[0] else -1.0
    idx = np.nonzero(sgn * (T - target) >= 0.0)[0]
    return float(t[idx[0]]) if idx.size else float("nan")


def temperatures(rows):
    """(time, T_e, T_lattice, T_spin) columns of observable rows."""
    rows = np.asarray(rows)
    return rows[:, COL_T], rows[:, COL_TE], rows[:, COL_TL], rows[:, COL_TSPIN0]
