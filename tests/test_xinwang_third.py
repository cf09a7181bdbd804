"""The third Xin-Wang inequality (Fig. `fig:filter`(b)): where on the child's interval it
must hold, checked by brute force on random face geometries (no GPU, no oracle code).

A child window on edge e of face (v0, v1, v2) is useless against T, the vertex of the
parent edge v0v1 that is not on e, when every point x of the child's interval is reached
more cheaply through T: d + |I x| > g_T + |T x|, i.e. f(x) = |I x| - |T x| exceeds
g_T - d everywhere on the interval.  The paper tests this at the end of the interval
nearer the vertex that e shares with the parent edge.  That is exact if f takes its
minimum over the interval there.  f has a single critical point on e's line, where x, I
and T are collinear (a maximum, f = |I T|, when T lies between I and x; a minimum,
f = -|I T|, when I does).  The interval is reached by the rays from I through the parent
window, between the rays through v0 and v1, and over it f falls towards the shared
vertex: sampled densely on random geometries below, the minimum over the interval is
always at that end.

The oracle and the propagation kernel test both ends (a window is dropped only when both
are dominated).  In exact arithmetic that is the same decision, because the end nearer
the shared vertex is the minimum; it differs only when rounding puts one end's test on
the wrong side of the margin.  These tests pin the exact-arithmetic fact by dense
sampling of each child's interval (points of e whose segment to I crosses the parent
edge inside the window)."""
import numpy as np

N_SAMPLES = 2001


def _child_interval(I, P, Q, A, B):
    """Points of segment P->Q reached by rays from I through [A, B] x {0} (the parent
    window), ordered from P to Q."""
    s = np.linspace(0.0, 1.0, N_SAMPLES)
    x = P[None, :] + s[:, None] * (Q - P)[None, :]
    # the segment I -> x crosses y = 0 at X (x has y >= 0, I has y < 0)
    X = I[0] + (x[:, 0] - I[0]) * (-I[1]) / (x[:, 1] - I[1])
    keep = (X >= A) & (X <= B)
    return x[keep]


def _faces(rng, n):
    """Random faces over the parent edge v0 = (0, 0), v1 = (1, 0), pseudo-sources below
    it (some nearly on its line, some far), windows on it (some ending on a vertex)."""
    for _ in range(n):
        v2 = np.array([rng.uniform(-3.0, 4.0), 10 ** rng.uniform(-3, 1)])
        I = np.array([rng.uniform(-10.0, 11.0), -(10 ** rng.uniform(-5, 1))])
        A, B = np.sort(rng.uniform(0.0, 1.0, 2))
        if rng.random() < 0.3:
            A = 0.0
        if rng.random() < 0.3:
            B = 1.0
        if B - A >= 1e-3:
            yield np.array([0.0, 0.0]), np.array([1.0, 0.0]), v2, I, A, B


def test_third_inequality_minimum_at_the_shared_vertex_end():
    rng = np.random.default_rng(20130513)
    checked = 0
    for v0, v1, v2, I, A, B in _faces(rng, 6000):
        # right child on v2 -> v1 (shares v1) against T = v0; left child on v0 -> v2
        # (shares v0) against T = v1
        for P, Q, T, shared_at_end in ((v2, v1, v0, True), (v0, v2, v1, False)):
            x = _child_interval(I, P, Q, A, B)
            if len(x) < 3:
                continue
            f = np.linalg.norm(x - I, axis=1) - np.linalg.norm(x - T, axis=1)
            near = f[-1] if shared_at_end else f[0]
            scale = np.linalg.norm(I - T) + 1.0
            assert f.min() >= near - 1e-12 * scale, (v2, I, A, B)
            checked += 1
    assert checked > 4000


def test_interior_minimum_when_I_lies_between_x_and_T():
    """The order the geometry excludes (I between x and T on one line) does put a minimum
    of f inside the line (f = -|I T| there): the sampling would see one if it existed."""
    I, T = np.array([0.3, -0.5]), np.array([0.6, -1.5])     # line T -> I meets y = 1 beyond I
    s = np.linspace(-3.0, 3.0, 60001)
    x = np.stack([s, np.ones_like(s)], axis=1)
    f = np.linalg.norm(x - I, axis=1) - np.linalg.norm(x - T, axis=1)
    j = int(np.argmin(f))
    assert 0 < j < len(s) - 1
    assert abs(f[j] + np.linalg.norm(I - T)) < 1e-6
