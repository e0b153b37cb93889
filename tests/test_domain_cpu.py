"""The triangular domain the 4ph kernels walk (host replica of their rule), checked against the
oracle's rectangular process lists (no GPU).

The summand of 4ph+- is symmetric under the partner swap (λ'', λ'''), that of ++ and -- under
(λ', λ'') when σ is fixed (Methodology, symmetric iteration region).  The kernels evaluate one
representative of each swapped pair with weight 2 and a self-paired point's ordered branch pairs:
  +-      q'' < q''' weight 2; q'' = q''' keeps j'' <= j''' (weight 2 if j'' < j''', else 1);
  ++, --  q'' > q'   weight 2; q'' = q'   keeps j'' >= j'   (weight 2 if j'' > j',   else 1).
+- takes its q'' <= q''' from a per-unit list; q''' = B - q'' (B = q + q') is an involution of the
mesh, so the list holds (N + F) / 2 points, F its fixed points (2 q'' = B per axis)."""
import numpy as np
import pytest

import oracle
from synth import morse_system

SIGNS = {2: (1, 1), 3: (1, -1), 4: (-1, -1)}


def representative_weight(ch, q1, j1, q2, j2, q3, j3):
    """Weight of a process in the domain, None if its swap represents it."""
    if ch == 3:
        if q2 != q3:
            return 2 if q2 < q3 else None
        return 2 if j2 < j3 else (1 if j2 == j3 else None)
    if q2 != q1:
        return 2 if q2 > q1 else None
    return 2 if j2 > j1 else (1 if j2 == j1 else None)


def q_index(c, mesh):
    return int(c[0] + mesh[0] * (c[1] + mesh[1] * c[2]))


@pytest.fixture(scope="module", params=[(3, 3, 3), (4, 2, 3)])
def prob(request):
    return oracle.Problem(*morse_system(seed=0), request.param)


@pytest.mark.parametrize("ch", [2, 3, 4])
def test_weights_recover_the_rectangular_set(prob, ch):
    """Σ weights over kept representatives = rectangular kept count, and every kept process is
    either a representative or the swap of a kept one."""
    P = prob
    nb, N, mesh = P.nb, P.nq, np.asarray(P.mesh)
    qc = oracle.q_coords(P.mesh)
    s1, s2 = SIGNS[ch]
    n_rep = 0
    for m0 in range(3, N * nb, 5):
        q0 = m0 // nb
        words = P.processes(ch, m0).tolist()
        tuples = set()
        for w in words:
            q1, j1, q2, j2, j3 = oracle.decode4(w, nb, N)
            q3 = q_index((qc[q0] + s1 * qc[q1] + s2 * qc[q2]) % mesh, P.mesh)
            tuples.add((q1, j1, q2, j2, q3, j3))
        total = 0
        for t in tuples:
            q1, j1, q2, j2, q3, j3 = t
            wt = representative_weight(ch, *t)
            if wt is None:
                swap = (q1, j1, q3, j3, q2, j2) if ch == 3 else (q2, j2, q1, j1, q3, j3)
                assert swap in tuples
                assert representative_weight(ch, *swap) == 2
            else:
                total += wt
                n_rep += 1
        assert total == len(tuples)
    assert n_rep > 0


@pytest.mark.parametrize("mesh", [(3, 3, 3), (4, 2, 3), (8, 8, 8), (5, 6, 4)])
def test_pm_list_length_closed_form(mesh):
    """|{q'' : q'' <= B - q''}| = (N + F) / 2 with F = Π_axes #{x : 2x = B_a mod n_a}."""
    qc = oracle.q_coords(mesh)
    n = np.asarray(mesh)
    N = int(np.prod(n))
    for B in qc[:: max(1, N // 37)]:
        q3 = [q_index((B - c) % n, mesh) for c in qc]
        listed = [q2 for q2 in range(N) if q2 <= q3[q2]]
        F = 1
        for a in range(3):
            F *= sum(1 for x in range(n[a]) if (2 * x - B[a]) % n[a] == 0)
        assert len(listed) == (N + F) // 2
        assert listed == sorted(listed)
