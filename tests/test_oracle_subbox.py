"""The sub-box form of the oracle used for the 512^3 blast: on a grid the oracle finishes in
seconds, the blast's result on the centred sub-box alone (periodic wrap, the full grid's cell
size) equals the full-grid result on those cells bit for bit, and the full grid is still the
uniform background outside them (section 4.1's step; the embedding argument is in
_helpers.blast_subbox_oracle)."""
import numpy as np

import oracle
from _helpers import blast_subbox_oracle, outer_layers_equal
from paper_1204_4779_gb300 import inputs


def test_box_generator_is_a_slice_of_the_full_field():
    full = inputs.blast_3d(64, radius_cells=8.0)
    box = inputs.blast_3d_box(64, 16, 32, radius_cells=8.0)
    assert np.array_equal(full[:, 16:48, 16:48, 16:48], box)


def test_subbox_run_equals_the_full_grid_run():
    n, lo, m, steps = 64, 10, 44, 25
    full = oracle.prim_to_cons(inputs.blast_3d(n, radius_cells=4.0), 1.4)
    Uf, tf, done, _ = oracle.run(full, 1.4, 0.4, steps, bc=(0, 0, 0), threads=oracle.max_threads())
    assert done == steps
    Ub, tb = blast_subbox_oracle(n, lo, m, steps, radius=4.0)
    assert tb == tf
    assert np.array_equal(Uf[:, lo:lo + m, lo:lo + m, lo:lo + m], Ub)
    bg = full[:, 0, 0, 0]
    outside = Uf.copy()
    outside[:, lo:lo + m, lo:lo + m, lo:lo + m] = bg.reshape(5, 1, 1, 1)
    assert np.all(outside == bg.reshape(5, 1, 1, 1))


def test_subbox_check_fails_when_the_box_is_too_small():
    """A sub-box the disturbance does reach is rejected, not silently wrapped."""
    try:
        blast_subbox_oracle(64, 24, 16, 25, radius=4.0)
    except AssertionError as e:
        assert "sub-box faces" in str(e)
    else:
        raise AssertionError("a 16^3 sub-box around a 25-step blast must be rejected")


def test_outer_layer_check():
    U = np.ones((5, 10, 10, 10))
    bg = np.ones(5)
    assert outer_layers_equal(U, bg, 4)
    U[2, 5, 5, 9] = 2.0
    assert not outer_layers_equal(U, bg, 4)
    U[2, 5, 5, 9] = 1.0
    U[2, 5, 5, 5] = 2.0  # the centre is not an outer layer
    assert outer_layers_equal(U, bg, 4)
