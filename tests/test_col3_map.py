"""The z-column 3D kernel's thread map and shared-memory accesses (host logic, no GPU).

The kernel (csrc/micro_fp32_3d_col.cuh) stores each z-plane with a row stride of
LD floats and gives thread t the tile (row y, column pair j) such that the 16
tiles of every half-warp have distinct (LD/2 * y + j) mod 16: 64-bit shared-memory
loads of a half-warp then hit 16 distinct bank pairs, for every offset the
stencil adds (a uniform shift). Half-warp g takes, for each residue r, the g-th
tile of residue r in row order; LD (>= N + 2, even) minimises the largest residue
class. This test restates that rule and checks, for every box size the kernel
takes and the smaller ones, that the map is a bijection onto the Ni x ceil(Ni/2)
tiles, that its inverse is the owner formula, and that every half-warp is
conflict-free.
"""


def _layout(N):
    Ni, P = N - 6, (N - 6 + 1) // 2
    best, best_ld = None, None
    for LD in range((N + 3) & ~1, N + 35, 2):
        L = LD // 2
        cnt = [0] * 16
        for y in range(Ni):
            for j in range(P):
                cnt[(L * y + j) & 15] += 1
        if best is None or max(cnt) < best:
            best, best_ld = max(cnt), LD
    return best_ld, best


def _tile(t, Ni, L):
    P, r, g = (Ni + 1) // 2, t & 15, t >> 4
    cnt = 0
    for y in range(Ni):
        j = (r - L * y) & 15
        if j < P:
            if cnt == g:
                return y, j
            cnt += 1
    return None


def _owner(y, j, Ni, L):
    P, r = (Ni + 1) // 2, (L * y + j) & 15
    return 16 * sum(1 for yy in range(y) if ((r - L * yy) & 15) < P) + r


def test_column_kernel_thread_map():
    for N in range(8, 33):
        LD, halfwarps = _layout(N)
        assert LD >= N + 2 and LD % 2 == 0
        Ni, L = N - 6, LD // 2
        NT = (16 * halfwarps + 31) // 32 * 32
        seen = {}
        for t in range(NT):
            tile = _tile(t, Ni, L)
            if tile is None:
                continue
            assert tile not in seen
            seen[tile] = t
            assert _owner(*tile, Ni, L) == t
        assert len(seen) == Ni * ((Ni + 1) // 2)
        for h in range(0, NT, 16):
            banks = [(L * y + j) & 15 for y, j in filter(None, (_tile(t, Ni, L) for t in range(h, h + 16)))]
            assert len(banks) == len(set(banks))
    # the 32^3 box: 338 tiles in 22 half-warps (352 threads), planes of 38-float rows
    assert _layout(32) == (38, 22)


def test_column_kernel_plane_reads_and_thread_order_arrays():
    """Every shared-memory access of the time loop stays inside its array. Thread t with
    tile (y, j) works at box row yb = 3 + y and box column xb0 = 3 + 2j, stored at plane
    offset rowoff = yb LD + xb0 + 1 (column x at offset x + 1): the y direction reads
    rowoff + m LD (+1) for m = -3 .. 3, the x direction rowoff - 4 .. rowoff + 5 on its
    own row; each of the kCol3S planes of a state array is one N x LD block. The
    per-thread arrays (m_init, H(m_init), H(W), the state's carry) are indexed by plane
    and thread, (k NT + t) 2 + h, inside kCol3S NT 2 floats per component."""
    S_MAX = 3
    for N in range(8, 33):
        LD, halfwarps = _layout(N)
        Ni, L = N - 6, LD // 2
        NT = (16 * halfwarps + 31) // 32 * 32
        PV = N * LD
        for t in range(NT):
            tile = _tile(t, Ni, L)
            if tile is None:
                continue
            y, j = tile
            yb, xb0 = 3 + y, 3 + 2 * j
            rowoff = yb * LD + xb0 + 1
            offs = [rowoff + m * LD + e for m in range(-3, 4) for e in (0, 1)]
            offs += [rowoff + e for e in range(-4, 6)]
            assert min(offs) >= 0 and max(offs) < PV, (N, t, tile)
            # the stores of the tile's own nodes stay in the interior rows and inside the row
            assert 3 <= yb <= N - 4 and xb0 + 2 < LD
            for k in range(S_MAX):
                for h in (0, 1):
                    io = (k * NT + t) * 2 + h
                    assert 0 <= io < S_MAX * NT * 2
