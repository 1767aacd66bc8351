"""Pins of Eq. (Wpart), the element cost model of the weighted partition.

Printed by the paper: the weight of a completely Out element is 1 and of a completely In element
0.  Fixed by the definition: an Intercepted element weighs its kept sub-cell points over 8 plus
T_s/T_v times its surface points over 8, and the surface part is linear in T_s/T_v.
"""
import numpy as np


def test_wpart_limits_and_cut_elements(small_sphere_oracle):
    w, m = small_sphere_oracle
    mk, _, _ = m.markers()
    sq = m.surface_points()
    ns = np.bincount(sq[:, 8].astype(np.int64), minlength=m.n_elem)
    W0 = m.wpart_weights(0.0)
    assert np.all(W0[(mk == 0)] == 1.0) and np.all(W0[mk == 1] == 0.0)
    cut = np.where(mk == 2)[0]
    n_cut_pts = np.array([m.cut_points(int(e)).shape[0] for e in cut])
    assert np.array_equal(W0[cut], n_cut_pts / 8.0)
    assert W0[cut].max() > 8.0                                   # some cut elements cost many Out ones
    W3 = m.wpart_weights(3.3)
    assert np.allclose(W3 - W0, 3.3 * ns / 8.0, rtol=0, atol=1e-12)
    # Out elements hosting no surface point stay at 1 whatever the ratio
    assert np.all(W3[(mk == 0) & (ns == 0)] == 1.0)
