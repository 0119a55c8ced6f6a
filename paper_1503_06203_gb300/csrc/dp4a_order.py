"""Generate the dp4a block order table of `dp4a_block` in xe_corr.cuh.

A chunk of 128 samples with kMmaK tensor-core k-steps runs its MMAs spread
evenly over (128 - 32 kMmaK) / 8 x 3 dp4a blocks (8 samples of one plane
each). A dp4a block on plane p accumulates into the registers that the MMAs
on plane p write, so it waits for those still in flight. The order of the
blocks is chosen by a seeded random search that minimises

    4 x (MMAs on the block's plane issued in the block)
  + 1 x (MMAs on the block's plane issued in the block before)
  + 1 x (consecutive blocks on the same plane)

over the orders with the same number of blocks per plane (seed 2 and 400,000
draws for chunks with 3 tensor-core k-steps, seed 11 and 150,000 draws for 2;
among orders of equal score the measured speeds still differ by a few tenths
of a percent, and these two measured best of those tried). Each table entry is
plane | (sample group << 2) in 5 bits, blocks 0-11 in the first word and
12-23 in the second. Run: python dp4a_order.py (prints the three words).
"""
import random

TC = 128  # samples per chunk


def mma_planes(mk):
    """Per block, the (plane, sub-tile) pairs of the MMAs issued in it."""
    mmas, blocks = mk * 6, (TC - 32 * mk) // 8 * 3
    return [{((m // 2) % 3, m & 1) for m in range(k * mmas // blocks, (k + 1) * mmas // blocks)}
            for k in range(blocks)]


def cost(order, planes):
    c = 0
    for k, p in enumerate(order):
        c += 4 * sum(1 for pl, _ in planes[k] if pl == p)
        if k:
            c += sum(1 for pl, _ in planes[k - 1] if pl == p) + (order[k - 1] == p)
    return c


def search(mk, seed=2, iters=400000):
    planes = mma_planes(mk)
    rng = random.Random(seed)
    items = [p for p in range(3) for _ in range(len(planes) // 3)]
    best, best_cost = None, None
    for _ in range(iters):
        rng.shuffle(items)
        c = cost(items, planes)
        if best_cost is None or c < best_cost:
            best, best_cost = list(items), c
    return best


def pack(order):
    seen = [0, 0, 0]
    words = [0, 0]
    for k, p in enumerate(order):
        words[k // 12] |= (p | (seen[p] << 2)) << (5 * (k % 12))
        seen[p] += 1
    return words


if __name__ == "__main__":
    w3 = pack(search(3))
    w2 = pack(search(2, seed=11, iters=150000))
    print(f"kMmaK 3: {w3[0]:#x}")
    print(f"kMmaK 2: {w2[0]:#x} {w2[1]:#x}")
