"""The staging schedule of the Jacobi kernel's three shared-memory slots
(CPU): block steps (I, I), (I, I+1), ..., (I, nb-1), (I+1, I+1), ...; before
each step's compute the one block the next step lacks is copied into the slot
that neither this step nor the next uses (empty slot first, then the lowest
block). This restates that rule and checks its invariants for every block
count the kernel meets: both blocks of a step are staged when it runs, a copy
never targets a slot in use, and every block pair is visited once per sweep.
"""
import pytest


def schedule(nb):
    held = [-1, -1, -1]

    def slot_of(b):
        return next((s for s in range(3) if held[s] == b), -1)

    held[0] = 0
    I = J = 0
    loads, visits = 1, []
    while True:
        nI, nJ = I, J + 1
        if nJ >= nb:
            nI, nJ = I + 1, I + 1
        more = nI < nb
        sX, sY = slot_of(I), slot_of(J)
        assert sX >= 0 and sY >= 0, "a step's blocks are staged"
        if more:
            need = nI if slot_of(nI) < 0 else (nJ if slot_of(nJ) < 0 else -1)
            if need >= 0:
                t = -1
                for s in range(3):
                    if s in (sX, sY) or held[s] in (nI, nJ):
                        continue
                    if t < 0 or held[s] < held[t]:
                        t = s
                assert t >= 0 and t not in (sX, sY), "the copy targets a free slot"
                held[t] = need
                loads += 1
        visits.append((min(I, J), max(I, J)))
        if not more:
            break
        I, J = nI, nJ
    return visits, loads


@pytest.mark.parametrize("nb", list(range(1, 33)))
def test_every_block_pair_once(nb):
    visits, loads = schedule(nb)
    assert sorted(visits) == [(i, j) for i in range(nb) for j in range(i, nb)]
    assert loads <= len(visits)  # at most one copy per step
