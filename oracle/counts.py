"""Number of MMBFs computed on the finest level (Table ntmmbfs).

Section 4 (MuMM): with piecewise-constant interface spaces on segments
(patches) of size H-bar and one Robin coefficient per segment, each leaf
needs one MMBF per interface patch on its boundary plus its particular
solution (the U-type and P-type responses of a patch differ only by the
factor -beta n.n^i, Eqs. 11Hhatbasisa/b with lambda = P - beta U n.n^i).
Section 5.1: the z direction is never cut, and H-bar_z = H_z.
"""


def mmbf_count(subdomains, ratio):
    """subdomains = (a, b, c) leaves per axis; ratio = (H/H-bar) per axis.
    Returns the total number of local solves on the finest level."""
    a, b, c = subdomains
    total = 0
    for k in range(c):
        for j in range(b):
            for i in range(a):
                patches = 0
                for axis, (idx, n) in enumerate(((i, a), (j, b), (k, c))):
                    tang = [ratio[d] for d in range(3) if d != axis]
                    per_face = tang[0] * tang[1]
                    patches += per_face * ((idx > 0) + (idx < n - 1))
                total += patches + 1
    return total
