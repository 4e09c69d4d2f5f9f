"""Pins of the oracle's agent actuation (Sec. 4 "Agent embodiment and action
space": stop, move_forward 0.25 m, turn_left / turn_right 10 degrees), each
against a fact that does not come from the oracle's own formula: closed-form
yaw quaternions, the 720-degree period of unit quaternions, the heading of a
yaw angle, and hand-built navigability grids."""
import math

import numpy as np
import pytest

from paper_1904_01201_b300 import workloads as wl

STOP, FWD, LEFT, RIGHT = 0, 1, 2, 3
OPEN = (np.float32(-10.0), np.float32(-10.0), np.float32(0.25), np.ones((80, 80), np.uint8))


def _pose(x, z, yaw, y=1.5):
    return np.r_[[x, y, z], wl.yaw_quat(np.array(yaw))].astype(np.float32)


def test_stop_is_identity(oracle_mod):
    p = _pose(1.3, -2.7, 0.77)
    out, moved = oracle_mod.actuate(p, STOP, OPEN)
    assert not moved and np.array_equal(out.view(np.uint32), p.view(np.uint32))


@pytest.mark.parametrize("yaw", [0.0, 0.3, 1.0, 2.5, -2.0, math.pi])
def test_turns_follow_closed_form_yaw(oracle_mod, yaw):
    """k left turns give the yaw quaternion of yaw + k*10 deg; right turns the
    negative angle (counter-clockwise seen from above is left, about +Y)."""
    for action, sign in ((LEFT, 1.0), (RIGHT, -1.0)):
        p = _pose(0.0, 0.0, yaw)
        for k in range(1, 19):
            p, moved = oracle_mod.actuate(p, action, OPEN)
            assert moved
            want = wl.yaw_quat(np.array(yaw + sign * math.radians(10.0) * k))
            # same double cover sign as the closed form for |angle| < 2 pi
            assert np.allclose(p[3:], want, atol=1e-6 * k), (action, k, p[3:], want)
            assert p[0] == 0.0 and p[1] == np.float32(1.5) and p[2] == 0.0


def test_full_circle_flips_quaternion_sign(oracle_mod):
    """36 turns of 10 degrees are one full turn: the unit quaternion comes back
    negated (q and -q are the same rotation); 72 turns restore it."""
    p0 = _pose(0.5, 0.5, 0.4)
    p = p0.copy()
    for k in range(72):
        p, _ = oracle_mod.actuate(p, LEFT, OPEN)
        if k == 35:
            assert np.allclose(p[3:], -p0[3:], atol=2e-5)
    assert np.allclose(p[3:], p0[3:], atol=4e-5)


@pytest.mark.parametrize("yaw", [0.0, 0.5, math.pi / 2, 2.0, -1.2])
def test_forward_moves_along_heading(oracle_mod, yaw):
    """The camera looks down -Z: at yaw th the horizontal heading is
    (-sin th, -cos th); one step moves 0.25 m along it, height unchanged."""
    p = _pose(1.0, 2.0, yaw)
    out, moved = oracle_mod.actuate(p, FWD, OPEN)
    assert moved
    want = np.array([1.0 - 0.25 * math.sin(yaw), 2.0 - 0.25 * math.cos(yaw)])
    assert np.allclose([out[0], out[2]], want, atol=2e-7 * 4)
    assert out[1] == p[1] and np.array_equal(out[3:], p[3:])


def test_forward_ignores_pitch(oracle_mod):
    """A pitched camera still steps 0.25 m horizontally along its yaw."""
    yaw, pitch = 0.7, 0.4
    qy = np.array([math.cos(yaw / 2), 0, math.sin(yaw / 2), 0])
    qx = np.array([math.cos(pitch / 2), math.sin(pitch / 2), 0, 0])
    w1, x1, y1, z1 = qy
    w2, x2, y2, z2 = qx
    q = np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                  w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    p = np.r_[[0.0, 1.5, 0.0], q].astype(np.float32)
    out, moved = oracle_mod.actuate(p, FWD, OPEN)
    assert moved and out[1] == p[1]
    assert np.allclose([out[0], out[2]], [-0.25 * math.sin(yaw), -0.25 * math.cos(yaw)], atol=1e-6)


def test_forward_refused_by_grid(oracle_mod):
    """Cells of 0.25 m from (0, 0): a step from the centre of cell (1, 3)
    facing -Z lands in cell (1, 2); blocking that cell (or leaving the grid)
    refuses the move and leaves the pose bit-identical."""
    grid = np.ones((4, 4), np.uint8)
    nav = (np.float32(0.0), np.float32(0.0), np.float32(0.25), grid)
    p = _pose(0.375, 0.875, 0.0)
    out, moved = oracle_mod.actuate(p, FWD, nav)
    assert moved and out[0] == np.float32(0.375) and out[2] == np.float32(0.625)
    grid[2, 1] = 0
    out, moved = oracle_mod.actuate(p, FWD, nav)
    assert not moved and np.array_equal(out.view(np.uint32), p.view(np.uint32))
    grid[2, 1] = 1
    grid[2, 0] = 0          # a neighbouring blocked cell does not matter
    assert oracle_mod.actuate(p, FWD, nav)[1]
    # leaving the grid through -Z from row 0 is refused
    p0 = _pose(0.375, 0.125, 0.0)
    assert not oracle_mod.actuate(p0, FWD, nav)[1]
    # a step ending exactly on a cell boundary belongs to the higher cell
    p1 = _pose(0.375, 1.0, 0.0)          # lands on z = 0.75 (row 3)
    grid[:] = 1
    grid[2, 1] = 0
    out, moved = oracle_mod.actuate(p1, FWD, nav)
    assert moved and out[2] == np.float32(0.75)
    grid[3, 1] = 0
    assert not oracle_mod.actuate(p1, FWD, nav)[1]


def test_unknown_action_rejected(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.actuate(_pose(0, 0, 0), 4, OPEN)


def test_random_walk_stays_navigable(oracle_mod):
    """A long random walk in a house: positions stay on navigable cells,
    the camera height is fixed and the quaternion stays unit length."""
    sc = wl.make_room(0)
    nav = wl.navmap(sc, 0.05)
    x0, z0, cell, grid = nav
    p = wl.navigable_poses(sc, nav, 1, 3)[0]
    rs = np.random.default_rng(5)
    refused = 0
    for a in rs.integers(0, 4, 600):
        q, moved = oracle_mod.actuate(p, int(a), nav)
        if a == FWD and not moved:
            refused += 1
        i = int(math.floor((float(q[0]) - float(x0)) / float(cell)))
        k = int(math.floor((float(q[2]) - float(z0)) / float(cell)))
        assert grid[k, i]
        assert q[1] == p[1]
        assert abs(float(np.linalg.norm(q[3:].astype(np.float64))) - 1.0) < 1e-6
        p = q
    assert refused > 0


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_turn_is_about_world_up_for_pitched_camera(oracle_mod):
    """Turning rotates about the world's vertical, not the camera's tilted up
    axis: yaw(th) pitch(ph) becomes yaw(th +- 10 deg) pitch(ph)."""
    yaw, pitch = 0.9, -0.35
    qx = np.array([math.cos(pitch / 2), math.sin(pitch / 2), 0, 0])
    p = np.r_[[0.0, 1.5, 0.0], _qmul(wl.yaw_quat(np.array(yaw)), qx)].astype(np.float32)
    for action, sign in ((LEFT, 1), (RIGHT, -1)):
        out, moved = oracle_mod.actuate(p, action, OPEN)
        want = _qmul(wl.yaw_quat(np.array(yaw + sign * math.radians(10.0))), qx)
        assert moved and np.allclose(out[3:], want, atol=1e-6), (action, out[3:], want)


def test_grid_bounds_on_every_side(oracle_mod):
    """Steps that leave a 3x3 grid through any side are refused, even when the
    memory around the grid holds navigable bytes."""
    big = np.ones((5, 5), np.uint8)
    for side, (x, z, yaw) in {"-z": (0.375, 0.125, 0.0), "+z": (0.375, 0.625, math.pi),
                              "-x": (0.125, 0.375, math.pi / 2), "+x": (0.625, 0.375, -math.pi / 2)}.items():
        flat = big.reshape(-1)
        grid = flat[6:15].reshape(3, 3)          # interior of a larger buffer of ones
        nav = (np.float32(0.0), np.float32(0.0), np.float32(0.25), grid)
        p = _pose(x, z, yaw)
        out, moved = oracle_mod.actuate(p, FWD, nav)
        assert not moved, side
        # one step in the opposite direction stays inside and is taken
        assert oracle_mod.actuate(_pose(x, z, yaw + math.pi), FWD, nav)[1], side


def test_turn_output_is_unit_from_non_unit_input(oracle_mod):
    """A pose quaternion off unit length by 5e-4 (accepted by the camera
    setup) turns into a unit quaternion and steps along its yaw heading.
    (Dividing the turned quaternion by its norm once more changes no float
    bit when the input was normalised: that reading has no separate pin.)"""
    p = _pose(0.0, 0.0, 1.1)
    p[3:] *= np.float32(1.0005)
    out, _ = oracle_mod.actuate(p, LEFT, OPEN)
    assert abs(float(np.linalg.norm(out[3:].astype(np.float64))) - 1.0) < 1e-6
    out, _ = oracle_mod.actuate(p, FWD, OPEN)
    assert np.allclose([out[0], out[2]], [-0.25 * math.sin(1.1), -0.25 * math.cos(1.1)], atol=1e-6)
