"""The tessellate tiling's schedule (paper Section 3.4, Fig. 6), checked on
the host through the library's own geometry code (no GPU needed):

* in 1D, stage 0 (triangles) updates each segment with the profile
  (0, 1, .., h, .., 1, 0) -- the paper's (0,1,2,3,4,3,2,1,0) for h = 4 on a
  segment of 2 h r + 1 points -- and stage 1 (inverted triangles) with the
  complement (h, .., 1, 0, 1, .., h), the paper's (4,3,2,1,0,1,2,3,4);
* in d dimensions there are d + 1 stages and their counts sum to h at every
  point (each point updated exactly once per level: no redundant work);
* stage 0 in d dimensions is the minimum over the axes of the 1D profile.
"""

import numpy as np
import pytest


def sgmod():
    import paper_2103_08825_gb300 as sg
    sg.load()
    return sg


def test_paper_1d_state_sequences():
    sg = sgmod()
    # three segments of 9 points, h = 4, r = 1 (Fig. 6: segments of 2 h r + 1)
    c = sg.stencil_tess_counts((27,), 1, 4, 9, True)
    tri = c[0][:9].tolist()
    assert tri == [0, 1, 2, 3, 4, 3, 2, 1, 0]
    # the halves of the inverted triangles around the segment's two cuts
    assert c[1][:9].tolist() == [4, 3, 2, 1, 0, 1, 2, 3, 4]
    assert np.all(c.sum(axis=0) == 4)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("r,h,tile,n", [(1, 4, 9, 40), (1, 4, 8, 27), (2, 3, 13, 50), (3, 2, 12, 12), (1, 6, 16, 97)])
def test_1d_profiles_and_sum(periodic, r, h, tile, n):
    sg = sgmod()
    c = sg.stencil_tess_counts((n,), r, h, tile, periodic)
    assert np.all(c.sum(axis=0) == h), c
    # stage 0 inside a segment [e, e'): min(h, distance to the segment's ends / r)
    m = 1 if n < 2 * tile else n // tile
    cuts = [i * tile for i in range(m)] + [n]
    exp = np.zeros(n, dtype=np.int64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        for x in range(a, b):
            exp[x] = min(h, (x - a) // r, (b - 1 - x) // r)
    np.testing.assert_array_equal(c[0], exp)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("shape,r,h,tile", [((40, 33), 1, 4, 9), ((64, 70), 2, 3, 16), ((21, 22, 23), 1, 2, 8)])
def test_nd_stages_partition_levels(shape, r, h, tile, periodic):
    sg = sgmod()
    d = len(shape)
    c = sg.stencil_tess_counts(shape, r, h, tile, periodic)
    assert c.shape[0] == d + 1                      # d + 1 stages
    assert np.all(c.sum(axis=0) == h)               # every point once per level
    # stage 0 (all axes shrinking) is the minimum of the 1D profiles
    prof = [sg.stencil_tess_counts((n,), r, h, tile, periodic)[0] for n in shape]
    grids = np.meshgrid(*prof, indexing="ij")
    np.testing.assert_array_equal(c[0], np.minimum.reduce(grids))


def test_segments_too_short_are_rejected():
    sg = sgmod()
    with pytest.raises(sg.StencilError):
        sg.stencil_tess_counts((30,), 2, 4, 10, False)   # 10 < 2 * 4 * 2
