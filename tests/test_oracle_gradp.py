"""Pins of the pressure term of the oracle's gradient criterion (Section 2.2: the
scaled-gradient test applied to density and pressure, as in the 3D case of
Section 4.2).

Each state below is built so that one reading of the test decides the outcome:
pressure taken from the conserved state (including the kinetic energy with its
factor 1/2), the pressure threshold separate from the density one, and
pressures of cells in absent blocks taken from the predicted conserved state.
"""
import numpy as np

import mrfv_inputs as mi
import oracle

G = 1.4


def _state(rho, vx, vy, p):
    """Conserved 2D level array (nv, ny, nx) from primitive fields."""
    E = p / (G - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
    return np.stack([rho, rho * vx, rho * vy, E])


def _flagged_children(left, right, eps_w, eps_p):
    """Level 0 of 4 x 2 blocks holds `left` for x < 1/2 and `right` beyond (each a
    (rho, vx, vy, p) tuple); returns the level-1 blocks the gradient criterion
    creates."""
    o = oracle.Oracle(2, 2, (4, 2, 1))
    o.init(mi.IC_UNIFORM, [1.0, 0.0, 0.0, 0.0, 1.0])
    o.set_exist(1, np.zeros(o.blocks_shape(1), np.uint8))
    ny, nx = o.cells_shape(0)
    x = np.broadcast_to(np.arange(nx)[None, :] >= nx // 2, (ny, nx))
    f = [np.where(x, r, l_) for l_, r in zip(left, right)]
    o.set_level(0, _state(*f))
    o.adapt(oracle.CRIT_GRAD, eps_w=eps_w, eta_tol=0.8, eps_p=eps_p)
    return o.get_exist(1)


def _jump_blocks(o_shape=(4, 8)):
    want = np.zeros(o_shape, np.uint8)
    want[:, 2:6] = 1  # children of level-0 blocks 1 and 2 (cells 8..23), which see the jump at cell 16
    return want


def test_pressure_jump_at_constant_density():
    left, right = (1.0, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, 1.2)
    assert not _flagged_children(left, right, eps_w=0.05, eps_p=0.0).any()
    assert np.array_equal(_flagged_children(left, right, eps_w=0.05, eps_p=0.05), _jump_blocks())


def test_contact_is_flagged_by_density_only():
    left, right = (1.0, 0.0, 0.0, 1.0), (0.5, 0.0, 0.0, 1.0)
    assert not _flagged_children(left, right, eps_w=10.0, eps_p=0.05).any()
    assert np.array_equal(_flagged_children(left, right, eps_w=0.05, eps_p=0.0), _jump_blocks())


def test_shear_changes_pressure_through_the_kinetic_energy():
    """Same density and total energy on both sides, tangential velocity 0 | 1:
    p = 0.4 (2.5 - 0.5 rho v^2) gives 1.0 | 0.8, a jump of 0.2 (0.4 without the
    factor 1/2, none without the kinetic term)."""
    o = oracle.Oracle(2, 2, (4, 2, 1))
    o.init(mi.IC_UNIFORM, [1.0, 0.0, 0.0, 0.0, 1.0])
    o.set_exist(1, np.zeros(o.blocks_shape(1), np.uint8))
    ny, nx = o.cells_shape(0)
    right = np.broadcast_to(np.arange(nx)[None, :] >= nx // 2, (ny, nx))
    Q = np.stack([np.ones((ny, nx)), np.zeros((ny, nx)), np.where(right, 1.0, 0.0), np.full((ny, nx), 2.5)])
    for eps_p, want in ((0.05, _jump_blocks()), (0.25, np.zeros((4, 8), np.uint8))):
        o.set_exist(1, np.zeros(o.blocks_shape(1), np.uint8))
        o.set_level(0, Q)
        o.adapt(oracle.CRIT_GRAD, eps_w=0.05, eta_tol=0.8, eps_p=eps_p)
        assert np.array_equal(o.get_exist(1), want), eps_p


def test_absent_neighbours_use_the_predicted_state():
    """Linear density and pressure at rest; on level 1 only the middle 2 x 2 blocks
    exist, so the cells one beyond them are predicted from level 0, which is
    exact for linear data.  The largest level-1 increment (the diagonal) is
    0.5/32 + 0.25/32 = 0.0234375: no level-1 flag at eps_p = 0.024, every
    existing level-1 block flagged at 0.023."""
    o = oracle.Oracle(2, 3, (2, 2, 1))
    o.init(mi.IC_UNIFORM, [1.0, 0.0, 0.0, 0.0, 1.0])

    def fields(l):
        ny, nx = o.cells_shape(l)
        xc = (np.arange(nx) + 0.5) / nx
        yc = (np.arange(ny) + 0.5) / ny
        X, Y = np.meshgrid(xc, yc)
        return _state(1.0 + 0.1 * X, 0 * X, 0 * X, 1.0 + 0.5 * X + 0.25 * Y)

    ex1 = np.zeros(o.blocks_shape(1), np.uint8)
    ex1[1:3, 1:3] = 1
    for eps_p, want in ((0.024, np.zeros_like(ex1)), (0.023, ex1)):
        o.set_exist(2, np.zeros(o.blocks_shape(2), np.uint8))
        o.set_exist(1, ex1)
        o.set_level(0, fields(0))
        o.set_level(1, fields(1))
        o.adapt(oracle.CRIT_GRAD, eps_w=1.0, eta_tol=0.8, eps_p=eps_p)
        assert np.array_equal(o.get_sig(1)[0], want), eps_p
