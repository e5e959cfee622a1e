"""Limited-memory BFGS oracle (TEST INFRASTRUCTURE only: ``tests/`` and the
CPU legs of ``bench.py`` may import it; the CUDA library never does).

The paper optimises most of its problems with SciPy's L-BFGS-B (Section 2.1)
on problems without bounds, keeping a history of 50 vector pairs (Section
3.1), i.e. limited-memory BFGS (Nocedal, Math. Comp. 35, 1980; Liu and
Nocedal, Math. Prog. 45, 1989).  The paper gives no algorithmic detail, so
the steps below are the textbook method with these readings (the same on
the GPU):

* search direction d_k = -H_k g_k by the two-loop recursion over the stored
  pairs (s_i, y_i), newest first, with H_k^0 = gamma_k I,
  gamma_k = s^T y / y^T y of the newest pair;
* the first direction is -g_0 and its first trial step 1 / ||g_0||_2 (a
  unit-length move); later first trials are t = 1;
* backtracking on the Armijo condition f(x + t d) <= f(x) + c1 t g^T d with
  c1 = 1e-4, halving t, at most 40 trials; if none passes, or g^T d >= 0,
  the run stops;
* after a step, the pair (s, y) = (x_new - x, g_new - g) is stored only if
  s^T y > 1e-12 y^T y (curvature), the oldest pair dropping out beyond m.

All vectors are float64 numpy arrays.  ``lbfgs`` takes a function returning
(f, g) and one returning f alone.
"""
from __future__ import annotations

import numpy as np

C1 = 1e-4
MAX_TRIALS = 40
CURV = 1e-12


def two_loop(g, pairs):
    """-H g for the pairs [(s, y, rho), ...] (oldest first), H0 = gamma I."""
    q = np.array(g, dtype=np.float64)
    if not pairs:
        return -q
    alpha = []
    for s, y, rho in reversed(pairs):
        a = rho * float(s @ q)
        alpha.append(a)
        q = q - a * y
    s, y, _ = pairs[-1]
    r = (float(s @ y) / float(y @ y)) * q
    for (s, y, rho), a in zip(pairs, reversed(alpha)):
        b = rho * float(y @ r)
        r = r + (a - b) * s
    return -r


def lbfgs(fg, f, x0, m, iterations):
    """Run L-BFGS from x0.  Returns (x, losses, done): losses[0] = f(x0),
    losses[k] = f after iteration k, done = iterations completed."""
    x = np.array(x0, dtype=np.float64)
    fx, g = fg(x)
    losses = [fx]
    pairs = []
    done = 0
    for k in range(iterations):
        d = two_loop(g, pairs)
        gd = float(g @ d)
        if not gd < 0.0:
            break
        t = 1.0 / float(np.sqrt(g @ g)) if k == 0 else 1.0
        accepted = False
        for _ in range(MAX_TRIALS):
            xt = x + t * d
            ft = f(xt)
            if ft <= fx + C1 * t * gd:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            break
        ft, gt = fg(xt)
        s = xt - x
        y = gt - g
        sy, yy = float(s @ y), float(y @ y)
        if sy > CURV * yy:
            pairs.append((s, y, 1.0 / sy))
            if len(pairs) > m:
                pairs.pop(0)
        x, g, fx = xt, gt, ft
        losses.append(fx)
        done += 1
    return x, losses, done


def explicit_inverse_hessian(pairs, n):
    """H from the BFGS inverse update applied to H0 = gamma I pair by pair
    (H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T): the dense matrix the
    two-loop recursion applies without forming it (for tests on tiny n)."""
    if not pairs:
        return np.eye(n)
    s, y, _ = pairs[-1]
    H = (float(s @ y) / float(y @ y)) * np.eye(n)
    eye = np.eye(n)
    for s, y, rho in pairs:
        V = eye - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H
