"""Host-side check of a base-level alignment: a CIGAR (uint32 length << 4 | BAM op)
is a valid alignment of query q to target t iff its '=' runs are equal bases, its
'X' bases differ, and together the operations consume both sequences exactly."""
EQ, DIFF, INS, DEL = 7, 8, 1, 2


def apply_cigar(q: bytes, t: bytes, ops) -> int:
    """Walk the CIGAR over q and t; returns its edit count, raises AssertionError
    where it is not a valid alignment."""
    i = j = cost = 0
    prev = None
    for o in ops:
        o = int(o)
        n, op = o >> 4, o & 15
        assert n > 0, "empty operation"
        assert op != prev, "adjacent operations of one kind are not merged"
        prev = op
        if op == EQ:
            assert q[i:i + n] == t[j:j + n], ("'=' over unequal bases", i, j, n)
            i += n
            j += n
        elif op == DIFF:
            assert i + n <= len(q) and j + n <= len(t)
            assert all(q[i + x] != t[j + x] for x in range(n)), ("'X' over equal bases", i, j)
            i += n
            j += n
            cost += n
        elif op == INS:
            i += n
            cost += n
        elif op == DEL:
            j += n
            cost += n
        else:
            raise AssertionError(f"unknown op {op}")
    assert i == len(q) and j == len(t), ("does not consume both sequences", i, len(q), j, len(t))
    return cost
