"""The slot algebra of in-place (AA-pattern) streaming, checked on a CPU model.

Even steps read a node's own slots [p][x] and write h*_p to [opp(p)][x]; odd
steps read [opp(p)][x - c_p] (or [p][x] when x - c_p is solid) and write h*_p to
[p][x + c_p] (or [opp(p)][x] when x + c_p is solid).  On a small box with a
wall and a pore this model checks that (a) every odd-step node writes exactly
the slots it read, and no slot is written twice -- the in-place update is
race-free -- and (b) after every step the post-collision values sit where the
pull scheme's next step (and the bead spread) expects them.  The collision is
any node-dependent map here; the GPU tests check the kernels themselves."""
import itertools

C = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0),
     (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
     (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
OPP = [0] + [p + 1 if p % 2 else p - 1 for p in range(1, 19)]


def _box():
    nx, ny, nz = 7, 5, 4
    solid = {(3, y, z) for y in range(ny) for z in range(nz)} - {(3, 2, 1), (3, 1, 2)}
    nodes = list(itertools.product(range(nx), range(ny), range(nz)))
    return (nx, ny, nz), solid, nodes


def _nb(n, p, s, dims):
    return tuple((n[a] + s * C[p][a]) % dims[a] for a in range(3))


def _collide(h, n):
    return [0.5 * v + 0.01 * p + 0.001 * sum(n) for p, v in enumerate(h)]


def test_inplace_slots_race_free_and_equal_to_pull():
    dims, solid, nodes = _box()
    fluid = [n for n in nodes if n not in solid]
    # pull scheme: post-collision values at [p][x]
    post = {(p, n): 0.1 * p + 0.01 * sum(n) + 0.001 * n[0] * p for n in fluid for p in range(19)}

    def pull_step(A):
        B = {}
        for n in fluid:
            h = [A[(OPP[p], n)] if _nb(n, p, -1, dims) in solid else A[(p, _nb(n, p, -1, dims))]
                 for p in range(19)]
            B.update({(p, n): v for p, v in enumerate(_collide(h, n))})
        return B

    # in place, starting from the swapped layout of the same post-collision values
    buf = {(OPP[p], n): v for (p, n), v in post.items()}
    A = dict(post)
    for step in range(4):
        odd = step % 2 == 0
        written = set()
        new = dict(buf)
        for n in fluid:
            if odd:
                reads = [(p, n) if _nb(n, p, -1, dims) in solid else (OPP[p], _nb(n, p, -1, dims))
                         for p in range(19)]
                writes = [(OPP[p], n) if _nb(n, p, 1, dims) in solid else (p, _nb(n, p, 1, dims))
                          for p in range(19)]
            else:
                reads = [(p, n) for p in range(19)]
                writes = [(OPP[p], n) for p in range(19)]
            assert set(writes) == set(reads)           # a node writes what it read
            assert not written & set(writes)           # no slot is written twice
            written |= set(writes)
            out = _collide([buf[r] for r in reads], n)
            new.update(dict(zip(writes, out)))
        buf = new
        A = pull_step(A)
        for (p, n), v in A.items():
            # where h*_p(n) must be after this step (the spread adds the bead source there)
            if odd:
                slot = (OPP[p], n) if _nb(n, p, 1, dims) in solid else (p, _nb(n, p, 1, dims))
            else:
                slot = (OPP[p], n)
            assert abs(buf[slot] - v) < 1e-12, (step, p, n)
