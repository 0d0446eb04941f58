"""The z-column 3D kernel's thread map (host logic, no GPU).

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
