"""The paper's subdivision cost model (Sec. 4), used to report the
model-optimal (g, r, B) next to the autotuner's measured choice.

Work (Sec. 4.1-4.2):

* exhaustive:  W_E = n^2 A                                   (Eq. 1-2)
* subdivision on a self-similar-density problem, Mandelbrot instance
  (Sec. 4.2.1), with G = g^2, R = r^2, tau = log_r(n / (g B)):
    W = sum_{i=0}^{tau-2} [4nA/(g r^i) + P lambda A + (1-P) n^2/(G R^i)] G R^i P^i
        + n^2 A P^(tau-1)
  i.e. per level: the perimeter query Q = 4nA/(g r^i), the subdivision
  cost S = lambda A with probability P and the terminal fill
  T = n^2/(G R^i) with probability 1 - P, over G R^i P^i regions; then
  the last level's per-pixel work L = n^2 A P^(tau-1).
* work-reduction factor  Omega = W_E / W  (Sec. 4.2.2; at most A).

Time on q multiprocessors of c cores (Sec. 4.3):

* exhaustive  T_Ex = ceil(n^2/(q c)) A
* SBR (one block of c cores per region), Delta[.] applied term by term
* MBR (several blocks per region for the fills and the last level)

lambda (the cost of one subdivision in units of A) is not given by the
paper for a GPU; :func:`fit_lambda` fits it, with a time scale, to measured
per-level times using :func:`level_terms`.

tau is real-valued in the paper; here the sums run over the levels
i = 0 .. floor(tau) - 2 and the powers of P use tau as given (a reading
of the paper's notation, stated in the design notes).  Only plain
arithmetic; nothing here runs on the GPU.
"""
import itertools
import math

POW2 = tuple(2 ** k for k in range(1, 11))  # the paper's search space {2, 4, ..., 1024}


def tau(n, g, r, B):
    """Subdivision depth of assumption iii: log_r(n / (g B))."""
    return math.log(n / (g * B), r)


def work_exhaustive(n, A):
    return float(n) * n * A


def work_ssd(n, g, r, B, P, A, lam):
    """W^M_SSD: total work of the Mandelbrot subdivision (Sec. 4.2.1)."""
    G, R = g * g, r * r
    t = tau(n, g, r, B)
    total = 0.0
    for i in range(0, int(math.floor(t)) - 1):  # i = 0 .. floor(tau) - 2
        q = 4.0 * n * A / (g * r ** i)
        s = P * lam * A
        fill = (1.0 - P) * n * n / (G * R ** i)
        total += (q + s + fill) * G * R ** i * P ** i
    return total + float(n) * n * A * P ** (t - 1.0)


def omega(n, g, r, B, P, A, lam):
    """Work-reduction factor W_E / W^M_SSD (Sec. 4.2.2)."""
    return work_exhaustive(n, A) / work_ssd(n, g, r, B, P, A, lam)


def _ceil(x):
    return float(math.ceil(x - 1e-9))


def time_exhaustive(n, A, q, c):
    """T_Ex = ceil(n^2 / (q c)) A (Sec. 4.3)."""
    return _ceil(n * n / (q * c)) * A


def time_sbr(n, g, r, B, P, A, lam, q, c):
    """T_SBR: single block per region (Sec. 4.3.1)."""
    G, R = g * g, r * r
    t = tau(n, g, r, B)
    total = 0.0
    for i in range(0, int(math.floor(t)) - 1):
        per_region = (_ceil(4.0 * n / (g * r ** i * c)) * A + P * lam * A
                      + (1.0 - P) * _ceil(n * n / (G * R ** i * c)))
        total += per_region * _ceil(G * R ** i / q) * P ** i
    last = (A * _ceil(n * n / (G * R ** (t - 1.0) * c)) * _ceil(G * R ** (t - 1.0) / q)
            * P ** (t - 1.0))
    return total + last


def time_mbr(n, g, r, B, P, A, lam, q, c):
    """T_MBR: multiple blocks per region for fills and the last level
    (Sec. 4.3.2)."""
    G, R = g * g, r * r
    S = lam * A
    t = tau(n, g, r, B)
    total = 0.0
    for i in range(0, int(math.floor(t)) - 1):
        total += (_ceil(4.0 * n / (g * r ** i * c)) * _ceil(G * R ** i / q) * A * P ** i
                  + _ceil(G * R ** i / q) * S * P ** (i + 1)
                  + _ceil(n * n * P ** i * (1.0 - P) / (q * c)))
    return total + A * _ceil(n * n / (q * c)) * P ** (t - 1.0)


def optimum(n, A, P, lam, q=152, c=128, scheme="sbr", space=POW2):
    """(g, r, B) minimising the model's time (scheme "sbr" or "mbr") or its
    work ("work") over `space`^3, among plans with tau >= 1."""
    best = None
    for g, r, B in itertools.product(space, space, space):
        if g * B > n or tau(n, g, r, B) < 1.0:
            continue
        if scheme == "sbr":
            v = time_sbr(n, g, r, B, P, A, lam, q, c)
        elif scheme == "mbr":
            v = time_mbr(n, g, r, B, P, A, lam, q, c)
        else:
            v = work_ssd(n, g, r, B, P, A, lam)
        if best is None or v < best[0]:
            best = (v, g, r, B)
    return best


def level_terms(n, g, r, A, q, c, regions, subdivs, leaves, levels):
    """The SBR time of Sec. 4.3.1 level by level, with the measured region
    and split counts in place of G R^i P^i and P: for level i with N_i
    regions of nominal side s_i = n / (g r^i) and split fraction
    P_i = splits_i / N_i,

        T_i = (ceil(4 s_i / c) A + (1 - P_i) ceil(s_i^2 / c)) ceil(N_i / q)
              + lambda * P_i A ceil(N_i / q),

    returned as the pair (a_i, b_i) with T_i = a_i + lambda b_i; then the
    last pass, A ceil(s_L^2 / c) ceil(N_leaf / q) with s_L the last level's
    side, as (a_L, 0)."""
    terms = []
    for i in range(levels):
        N = float(regions[i])
        if N <= 0:
            terms.append((0.0, 0.0))
            continue
        s_i = n / (g * float(r) ** i)
        Pi = subdivs[i] / N
        waves = _ceil(N / q)
        a = (_ceil(4.0 * s_i / c) * A + (1.0 - Pi) * _ceil(s_i * s_i / c)) * waves
        terms.append((a, Pi * A * waves))
    s_L = n / (g * float(r) ** (levels - 1))
    terms.append((A * _ceil(s_L * s_L / c) * _ceil(float(leaves) / q) if leaves else 0.0, 0.0))
    return terms


def fit_lambda(ms, terms):
    """Least-squares fit of ms_i = kappa (a_i + lambda b_i) over the levels
    and the last pass, kappa >= 0 and lambda >= 0.  ms: measured times in the
    order of level_terms.  Returns (kappa in ms per model time unit,
    lambda)."""
    import numpy as np
    X = np.array([[a, b] for a, b in terms], dtype=np.float64)
    y = np.array(ms, dtype=np.float64)
    sol, *_ = np.linalg.lstsq(X, y, rcond=None)
    kappa, mu = float(sol[0]), float(sol[1])
    if mu < 0.0 or kappa <= 0.0:
        # refit with lambda = 0 (kappa alone)
        mu = 0.0
        den = float((X[:, 0] ** 2).sum())
        kappa = float((X[:, 0] * y).sum() / den) if den > 0 else 0.0
    return kappa, (mu / kappa if kappa > 0 else 0.0)


def estimate_p(stats):
    """Subdivision probability from measured per-level counts: splits over
    regions evaluated, pooled over the levels that may split."""
    regs = stats["regions_per_level"]
    subs = stats["subdivisions_per_level"]
    num = sum(subs[:-1])
    den = sum(regs[:-1])
    return num / den if den else 0.0
