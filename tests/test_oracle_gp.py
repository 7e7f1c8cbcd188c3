"""Pins of the oracle's machine-code controller (Sec. IV, Table I) against hand-worked traces:
every opcode, the accumulator's 8-bit wrap, the program counter's wrap after address 31, the
5-degree motor steps and their saturation, and the controller driving the joint updates of a
full step."""
import math

import numpy as np
import pytest

from oracle.oracle import GP_LEN, Oracle, gp_run
from paper_2411_05799_gb300 import scenes


def op(cmd, x=0):
    """Opcode byte: 3-bit command (Table I order) and 5-bit value."""
    return (cmd << 5) | x


LEFT, RIGHT, READ, LOAD, JUMP, NOT, INC, DEC = range(8)


def prog(*codes, fill=op(LOAD, 0)):
    p = np.full(GP_LEN, fill, np.uint8)
    p[:len(codes)] = codes
    return p


def test_accumulator_commands():
    # load 5, inc, inc, dec -> 6
    pc, acc, _ = gp_run(prog(op(LOAD, 5), op(INC), op(INC), op(DEC)), 0, 0, [], 0, 4)
    assert (pc, acc) == (4, 6)
    # load 0, dec -> 255 (8-bit wrap), inc -> 0, not -> 255, not -> 0
    assert gp_run(prog(op(LOAD, 0), op(DEC)), 0, 0, [], 0, 2)[1] == 255
    assert gp_run(prog(op(LOAD, 0), op(DEC), op(INC)), 0, 0, [], 0, 3)[1] == 0
    assert gp_run(prog(op(LOAD, 0), op(NOT)), 0, 0, [], 0, 2)[1] == 255
    assert gp_run(prog(op(LOAD, 12), op(NOT)), 0, 0, [], 0, 2)[1] == 243
    assert gp_run(prog(op(LOAD, 31), op(NOT), op(NOT)), 0, 0, [], 0, 3)[1] == 31


def test_read_sensor_gives_the_foot_bit():
    sensors = 0b101010
    for bit in range(8):
        _, acc, _ = gp_run(prog(op(READ, bit)), 0, 7, [], sensors, 1)
        assert acc == (sensors >> bit) & 1


def test_jump_if_true():
    # load 0; jump 9 (not taken: pc 2); load 1; jump 9 (taken: pc 9)
    code = prog(op(LOAD, 0), op(JUMP, 9), op(LOAD, 1), op(JUMP, 9))
    assert gp_run(code, 0, 0, [], 0, 2)[0] == 2
    assert gp_run(code, 0, 0, [], 0, 4)[0] == 9
    # a two-instruction loop at addresses 5-6 keeps the counter there
    code = prog(op(LOAD, 1), fill=op(LOAD, 1))
    code[5], code[6] = op(LOAD, 3), op(JUMP, 5)
    pc, acc, _ = gp_run(code, 5, 0, [], 0, 33)
    assert (pc, acc) == (6, 3)


def test_program_counter_wraps_and_budget():
    # 32 loads from address 20: 12 to the end, then 0..19; the last one executed is address 19
    code = np.array([op(LOAD, i % 32) for i in range(32)], np.uint8)
    pc, acc, _ = gp_run(code, 20, 0, [], 0, 32)
    assert (pc, acc) == (20, 19)
    pc, acc, _ = gp_run(code, 31, 0, [], 0, 1)
    assert (pc, acc) == (0, 31)


def test_motor_steps_saturate_and_missing_motors_are_ignored():
    k = np.zeros(3, np.int8)
    # right 0 three times, left 2 twice, right 17 (no such motor)
    code = prog(op(RIGHT, 0), op(RIGHT, 0), op(RIGHT, 0), op(LEFT, 2), op(LEFT, 2), op(RIGHT, 17))
    _, _, k = gp_run(code, 0, 0, k, 0, 6)
    assert list(k) == [3, 0, -2]
    # 32 x right 1 from 30: saturates at +36; 32 x left 1 from -20: saturates at -36
    code = np.full(GP_LEN, op(RIGHT, 1), np.uint8)
    assert list(gp_run(code, 0, 0, [0, 30, 0], 0, 32)[2]) == [0, 36, 0]
    code = np.full(GP_LEN, op(LEFT, 1), np.uint8)
    assert list(gp_run(code, 0, 0, [0, -20, 0], 0, 32)[2]) == [0, -36, 0]


def test_controller_drives_the_joint_updates():
    """A program that moves motor 0 right once and then loops on addresses 1-2: after the first
    joint update joint 0 stands at exactly 5 degrees and stays there; every other joint at 0.
    A second program moves motor 3 left on every pass while foot sensor 0 reads 1 (the hexapod
    stands on its feet): its target falls 5 degrees per executed move until the joint limit."""
    b = scenes.hexapod_batch(2, seed_key=1)
    p0 = prog(op(RIGHT, 0), op(LOAD, 1), op(JUMP, 1))
    # read sensor 0; jump to 4 if set; load 1; jump 0; left 3; load 1; jump 0
    p1 = prog(op(READ, 0), op(JUMP, 4), op(LOAD, 1), op(JUMP, 0), op(LEFT, 3), op(LOAD, 1), op(JUMP, 0))
    o = Oracle(b, gp_programs=np.stack([p0, p1]))
    K = b.joint_update_steps
    o.step(1)                                    # step 0: the first joint update
    jo = b.joint_off
    th0 = o.theta[jo[0]:jo[1]]
    assert th0[0] == pytest.approx(math.radians(5.0), abs=1e-15)
    assert np.all(th0[1:] == 0.0)
    assert o.gp_k[jo[0]] == 1
    o.step(3 * K)                                # three more joint updates, then a few steps
    assert o.theta[jo[0]] == pytest.approx(math.radians(5.0), abs=1e-15)
    assert int(o.gp_pc[0]) in (1, 2)
    # scene 1: feet start 1 cm above ground, so the first update reads 0 and moves nothing
    k3 = int(o.gp_k[jo[1] + 3])
    assert k3 <= 0
    lo = float(b.lo[b.link_off[1] + 3 + 1])
    assert o.theta[jo[1] + 3] == pytest.approx(max(k3 * math.radians(5.0), lo), abs=1e-12)
    o.step(20 * K)                               # standing: the foot bit is set, motor 3 keeps moving
    assert o.gp_k[jo[1] + 3] < k3
    assert o.theta[jo[1] + 3] >= lo - 1e-12
