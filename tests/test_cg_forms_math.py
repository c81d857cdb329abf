"""The two CG iteration forms of the solver are the same CG on the normal
equations A^+ A x = A^+ b (Sec. 5.1 solves; the least-squares form that
tracks r = b - A x and s = A^+ r):

* five launches: s is carried by s <- s - alpha A^+ q, q = A p;
* six launches: s = A^+ r is recomputed from the updated r.

In exact arithmetic both produce the same x, r, s, p at every iteration,
which is what lets the solver time them on real iterations and switch form
at an iteration boundary.  Checked in FP64 on a small dense non-Hermitian
system, for each form alone and for a switch of form every few iterations,
together with the properties of the iteration (the residual norm falls
monotonically and the solution is reached)."""
import numpy as np
import pytest


def _system(n=48, seed=0):
    rng = np.random.default_rng(seed)
    g = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
    A = np.eye(n) + 0.6 * g
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def _start(A, b):
    r = b.copy()
    s = A.conj().T @ r
    return {"x": np.zeros_like(b), "r": r, "s": s, "p": s.copy(), "gamma": np.vdot(s, s).real}


def _iterate(A, st, form):
    q = A @ st["p"]
    alpha = st["gamma"] / np.vdot(q, q).real
    x = st["x"] + alpha * st["p"]
    r = st["r"] - alpha * q
    if form == "five":
        s = st["s"] - alpha * (A.conj().T @ q)
    else:
        s = A.conj().T @ r
    gamma = np.vdot(s, s).real
    p = s + (gamma / st["gamma"]) * st["p"]
    return {"x": x, "r": r, "s": s, "p": p, "gamma": gamma}


def _run(A, b, forms):
    st = _start(A, b)
    out = []
    for f in forms:
        st = _iterate(A, st, f)
        out.append(st)
    return out


@pytest.mark.parametrize("pattern", ["six", "alternate", "blocks"])
def test_forms_give_the_same_iterates(pattern):
    A, b = _system()
    n = 14
    five = _run(A, b, ["five"] * n)
    if pattern == "six":
        other = _run(A, b, ["six"] * n)
    elif pattern == "alternate":
        other = _run(A, b, ["five" if k % 2 else "six" for k in range(n)])
    else:
        # the solver's timing order: one of each, then blocks five, six, six, five
        other = _run(A, b, ["five", "six"] + ["five"] * 3 + ["six"] * 6 + ["five"] * 3)
    for k in range(n):
        for key in ("x", "r", "s", "p"):
            a, c = five[k][key], other[k][key]
            assert np.linalg.norm(a - c) <= 1e-10 * np.linalg.norm(a), (pattern, k, key)


def test_the_carried_normal_residual_is_the_normal_residual():
    A, b = _system(seed=3)
    for st in _run(A, b, ["five"] * 20):
        s_true = A.conj().T @ st["r"]
        assert np.linalg.norm(st["s"] - s_true) <= 1e-10 * np.linalg.norm(s_true)
        assert np.linalg.norm(st["r"] - (b - A @ st["x"])) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("form", ["five", "six"])
def test_residual_falls_monotonically_and_the_solution_is_reached(form):
    A, b = _system(seed=5)
    hist = _run(A, b, [form] * 60)
    norms = [np.linalg.norm(st["r"]) for st in hist]
    # CG on the normal equations minimises |b - A x| over the Krylov space
    # (checked above the FP64 rounding floor, where the carried s of the
    # five-launch form stops following A^+ r)
    floor = 1e-12 * np.linalg.norm(b)
    assert all(n1 <= n0 * (1 + 1e-12) for n0, n1 in zip(norms, norms[1:]) if n1 > floor)
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(hist[-1]["x"] - x) <= 1e-8 * np.linalg.norm(x)


def test_a_dropped_term_in_the_five_launch_update_is_caught():
    """Planted mistake: s <- s - alpha A q (A instead of A^+) drifts from the
    six-launch iterates within a few iterations."""
    A, b = _system(seed=7)
    st5 = st6 = _start(A, b)
    worst = 0.0
    for _ in range(6):
        q = A @ st5["p"]
        alpha = st5["gamma"] / np.vdot(q, q).real
        bad = dict(st5)
        bad["x"] = st5["x"] + alpha * st5["p"]
        bad["r"] = st5["r"] - alpha * q
        bad["s"] = st5["s"] - alpha * (A @ q)
        g = np.vdot(bad["s"], bad["s"]).real
        bad["p"] = bad["s"] + (g / st5["gamma"]) * st5["p"]
        bad["gamma"] = g
        st5 = bad
        st6 = _iterate(A, st6, "six")
        worst = max(worst, np.linalg.norm(st5["x"] - st6["x"]) / np.linalg.norm(st6["x"]))
    assert worst > 1e-3
