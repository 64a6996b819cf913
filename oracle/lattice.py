"""Square L x L lattice with periodic boundaries (Sec. 6.1, "Physical systems").

Site (x, y), 0 <= x, y < L, has index y*L + x.

Bond order (fixes the order of every connected-configuration list):
site-major over i = 0..N-1, then direction
    0: (i, i + x)        nearest neighbour
    1: (i, i + y)        nearest neighbour
    2: (i, i + x + y)    next-nearest neighbour
    3: (i, i + x - y)    next-nearest neighbour
all coordinates mod L. The J1-J2 model of Eq. (2) uses all four directions,
the t-J model of Eq. (3) only the first two.
"""

NN_DIRS = ((1, 0), (0, 1))
NNN_DIRS = ((1, 1), (1, -1))


def site(x, y, L):
    return (y % L) * L + (x % L)


def coords(i, L):
    return i % L, i // L


def bonds(L, with_nnn):
    """List of (i, j, is_nnn) in the bond order above."""
    dirs = NN_DIRS + (NNN_DIRS if with_nnn else ())
    out = []
    for i in range(L * L):
        x, y = coords(i, L)
        for k, (dx, dy) in enumerate(dirs):
            out.append((i, site(x + dx, y + dy, L), k >= 2))
    return out


def snake_position(i, L):
    """Position of site i along the snake (boustrophedon) path.

    Row y is traversed left to right when y is even and right to left when y
    is odd. This is the mode ordering of the Jordan-Wigner encoding used for
    the fermion signs of Eq. (3).
    """
    x, y = coords(i, L)
    return y * L + (x if y % 2 == 0 else L - 1 - x)


def sublattice_a(i, L):
    """True on the (x + y) even sublattice (used by the optional sign rule)."""
    x, y = coords(i, L)
    return (x + y) % 2 == 0
