"""The host-side CIGAR checker used by the GPU base-level alignment tests, pinned
on alignments written by hand and on alignments built from known edit scripts."""
import pytest

import oracle
from cigar_check import DEL, DIFF, EQ, INS, apply_cigar


def c(*ops):
    return [(n << 4) | op for n, op in ops]


def test_hand_alignments():
    # ACGT vs AGT: the C is a query base absent from the target
    assert apply_cigar(b"ACGT", b"AGT", c((1, EQ), (1, INS), (2, EQ))) == 1
    assert apply_cigar(b"AGT", b"ACGT", c((1, EQ), (1, DEL), (2, EQ))) == 1
    assert apply_cigar(b"ACGT", b"AGGT", c((1, EQ), (1, DIFF), (2, EQ))) == 1
    assert apply_cigar(b"", b"", []) == 0
    assert apply_cigar(b"AC", b"", c((2, INS))) == 2


@pytest.mark.parametrize("q,t,ops", [
    (b"ACGT", b"AGT", c((1, EQ), (1, DIFF), (2, EQ))),        # does not consume t exactly
    (b"ACGT", b"AGGT", c((4, EQ))),                           # '=' over a mismatch
    (b"ACGT", b"ACGT", c((1, EQ), (1, DIFF), (2, EQ))),       # 'X' over equal bases
    (b"ACGT", b"ACGT", c((2, EQ), (2, EQ))),                  # unmerged runs
    (b"ACGT", b"ACGT", c((0, EQ), (4, EQ))),                  # empty operation
])
def test_rejects_invalid(q, t, ops):
    with pytest.raises(AssertionError):
        apply_cigar(q, t, ops)


def test_edit_scripts_match_levenshtein_bound():
    """A CIGAR built from an edit script costs the script's length, which bounds the
    Levenshtein distance from above (equal when the script is short and spaced)."""
    import random
    rnd = random.Random(5)
    for _ in range(200):
        t = bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(1, 60)))
        q, ops, cost = bytearray(), [], 0
        for b in t:
            r = rnd.random()
            if r < 0.05:
                ops.append(DEL)
                cost += 1
            elif r < 0.10:
                q.append([x for x in b"ACGT" if x != b][rnd.randint(0, 2)])
                ops.append(DIFF)
                cost += 1
            else:
                q.append(b)
                ops.append(EQ)
            if rnd.random() < 0.05:
                q.append(rnd.choice(b"ACGT"))
                ops.append(INS)
                cost += 1
        runs = []
        for op in ops:
            if runs and runs[-1][1] == op:
                runs[-1][0] += 1
            else:
                runs.append([1, op])
        assert apply_cigar(bytes(q), t, c(*runs)) == cost
        assert oracle.levenshtein(bytes(q), t) <= cost
