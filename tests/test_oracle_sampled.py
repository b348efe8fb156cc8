"""Pins of oracle/sampled.py: the continuous box spline by exact polygon
areas, and the equality of the paper's route (running sums interpolated by
beta_b, then differences) with the sampled continuous box spline."""
import math
import random
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import kernels, params
from oracle import sampled as sp
from oracle.rounding import quantize
from workloads import synth

ONES = (Fr(1),) * 4


def test_grid_box_spline_values():
    # the box spline of the four unit steps (Zwart-Powell element): 1/2 at
    # its centre (1/2, 3/2), 1/8 one step away along the axes, 0 at the
    # octagon's corners
    assert sp.beta(Fr(1, 2), Fr(3, 2), ONES) == Fr(1, 2)
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        assert sp.beta(Fr(1, 2) + dx, Fr(3, 2) + dy, ONES) == Fr(1, 8)
    assert sp.beta(Fr(-1), Fr(3, 2), ONES) == 0 and sp.beta(Fr(2), Fr(3, 2), ONES) == 0


def test_partition_of_unity():
    # the shifts of beta_b by the lattice sum to one everywhere
    rng = random.Random(0)
    for _ in range(40):
        x = (Fr(rng.randrange(0, 1024), 1024), Fr(rng.randrange(0, 1024), 1024))
        s = sum(sp.beta(x[0] - m1, x[1] - m2, ONES) for m1 in range(-3, 4) for m2 in range(-4, 4))
        assert s == 1


def test_axis_boxes_reduce_to_a_rectangle():
    # with the diagonal boxes short, beta_a tends to the rectangle
    # 1/(l1 l3) on its support (here the diagonal parts are 1/512 long)
    lam = (Fr(3), Fr(1, 512), Fr(2), Fr(1, 512))
    assert sp.beta(Fr(3, 2), Fr(1), lam) == Fr(1, 6)
    assert sp.beta(Fr(4), Fr(1), lam) == 0


def test_unit_mass_symmetry_and_covariance():
    lam = (Fr(5, 2), Fr(3, 2), Fr(7, 4), Fr(1, 2))
    h = Fr(1, 8)
    tx = (lam[0] + lam[1] - lam[3]) / 2
    ty = (lam[1] + lam[2] + lam[3]) / 2
    mass = Fr(0)
    m2 = np.zeros((2, 2))
    for i in range(-40, 41):
        for j in range(-40, 41):
            y = (tx + (i + Fr(1, 2)) * h, ty + (j + Fr(1, 2)) * h)
            b = sp.beta(y[0], y[1], lam)
            if not b:
                continue
            # symmetric about the centre
            assert b == sp.beta(2 * tx - y[0], 2 * ty - y[1], lam)
            mass += b * h * h
            v = np.array([float(y[0] - tx), float(y[1] - ty)])
            m2 += float(b * h * h) * np.outer(v, v)
    assert abs(float(mass) - 1) < 2e-3
    want = sum(float(l) ** 2 / 12 * np.outer(d, d) for l, d in zip(lam, ([1, 0], [1, 1], [0, 1], [-1, 1])))
    assert np.allclose(m2, want, atol=0.02)


def test_pieces_are_quadratic_on_the_four_directional_mesh():
    # third differences vanish inside a triangle of the criss-cross mesh
    rng = random.Random(1)
    for _ in range(30):
        # a point inside a triangle: keep clear of the lines x, y, x +- y in Z
        cx, cy = rng.randrange(-1, 2), rng.randrange(0, 3)
        base = (Fr(cx) + Fr(rng.randrange(30, 34), 64), Fr(cy) + Fr(rng.randrange(5, 9), 64))
        for d in ((Fr(1, 512), 0), (0, Fr(1, 512)), (Fr(1, 512), Fr(1, 1024))):
            v = [sp.beta(base[0] + k * d[0], base[1] + k * d[1], ONES) for k in range(4)]
            assert v[3] - 3 * v[2] + 3 * v[1] - v[0] == 0


def test_weights_are_integers_over_2_to_23():
    rng = random.Random(2)
    for _ in range(200):
        x = (Fr(rng.randrange(-1024, 2048), 1024), Fr(rng.randrange(0, 3072), 1024))
        w = sp.beta(x[0], x[1], ONES) * (1 << sp.WEIGHT_BITS)
        assert w.denominator == 1


@pytest.mark.parametrize("boundary", [0, 2])
def test_paper_route_equals_the_sampled_box_spline(boundary):
    # the running sums interpolated by beta_b and differenced at the
    # continuous offsets give exactly sum_m f(m) beta_a(p + tau - m)
    H, W = 9, 11
    f = synth.random_integer_image(H, W, seed=3, lo=-20, hi=20).astype(np.float64)
    fq = quantize(f, 0, as_object=True)
    rng = random.Random(4 + boundary)
    for _ in range(6):
        Lq = np.array([rng.randrange(1, 1400) for _ in range(4)])
        R = int(sp.reach(Lq)) + 1
        y, x = rng.randrange(H), rng.randrange(W)
        a = sp.exact_value(fq, Lq, boundary, y, x)
        b = sp.paper_route_value(fq, Lq, boundary, y, x, R)
        assert a == b


def test_constant_image_and_steps():
    # unit mass: a constant image stays constant up to the sampling of
    # beta_a; the quantised steps follow the float32 scale solve
    H, W = 20, 20
    cov = synth.constant_cov_field(H, W, 6.0, 1.0, 4.0)
    Lq, fl = sp.lambdas_q(cov[0], cov[1], cov[2])
    A, _ = params.solve_scales_f32(np.float32(6.0), np.float32(1.0), np.float32(4.0), 1)
    want = [round(math.sqrt(float(A[k]) / (1, 2, 1, 2)[k]) * 512) for k in range(4)]
    assert [int(v) for v in Lq[:, 0, 0]] == want
    f = np.full((H, W), 3.0)
    out = sp.filter_sampled(f, cov, kernels.REPLICATE, 10, out_dtype=np.float64, pixels=[(10, 10)])
    assert abs(out[(10, 10)] - 3.0) < 0.05


def test_second_set_grid_box_spline():
    # beta'_b: unit mass, partition of unity over the lattice, symmetric about
    # its centre (0, 3) under the reflections of the square, zero outside
    # its octagon (the zonotope of the four steps) and positive inside
    rng = random.Random(5)
    for _ in range(12):
        x = (Fr(rng.randrange(0, 64), 64), Fr(rng.randrange(0, 64), 64))
        assert sum(sp.beta_k(x[0] - m1, x[1] - m2, ONES) for m1 in range(-4, 5) for m2 in range(-7, 2)) == 1
    for _ in range(40):
        a, b = Fr(rng.randrange(-190, 191), 64), Fr(rng.randrange(-190, 191), 64)
        v = sp.beta_k(a, 3 + b, ONES)
        for a2, b2 in ((b, a), (-a, b), (a, -b), (-b, -a)):
            assert sp.beta_k(a2, 3 + b2, ONES) == v
    # the octagon: |x| + ... ; vertices of sum_k [0, e_k] include (0, 0), (2, 1), (3, 3), (0, 6)
    assert sp.beta_k(Fr(0), Fr(0), ONES) == 0 and sp.beta_k(Fr(0), Fr(6), ONES) == 0
    assert sp.beta_k(Fr(0), Fr(3), ONES) > 0 and sp.beta_k(Fr(5, 2), Fr(3), ONES) > 0
    assert sp.beta_k(Fr(3), Fr(3), ONES) == 0 and sp.beta_k(Fr(-3), Fr(3), ONES) == 0


def test_second_set_weights_are_integers_over_491520():
    rng = random.Random(6)
    for _ in range(300):
        x = (Fr(rng.randrange(-192, 193), 64), Fr(rng.randrange(0, 385), 64))
        assert (sp.beta_k(x[0], x[1], ONES) * sp.WEIGHT_DEN_K).denominator == 1


@pytest.mark.parametrize("boundary", [0, 2])
def test_second_set_paper_route_equals_the_sampled_box_spline(boundary):
    # Algorithm 3 as printed (running sums along (2,1), (1,2), (-1,2), (-2,1),
    # interpolation by beta'_b, the 16-tap differences) is exactly the
    # sampled beta'_a
    H, W = 7, 8
    f = synth.random_integer_image(H, W, seed=7, lo=-9, hi=9).astype(np.float64)
    fq = quantize(f, 0, as_object=True)
    rng = random.Random(8 + boundary)
    for _ in range(4):
        Lq = np.array([rng.randrange(1, 90) for _ in range(4)])
        R = int(sp.reach_k(Lq)) + 1
        y, x = rng.randrange(H), rng.randrange(W)
        a = sp.exact_value_k(fq, Lq, boundary, y, x)
        assert a == sp.paper_route_value_k(fq, Lq, boundary, y, x, R)
        sp.accumulator_k(a, Lq)   # integral


def test_second_set_covariance():
    # the continuous beta'_a has covariance sum_k lambda_k^2 e_k e_k^T / 12
    lam = (Fr(3, 2), Fr(1), Fr(5, 4), Fr(3, 4))
    h = Fr(1, 6)
    tx = sum(l * e[0] for l, e in zip(lam, sp._E)) / 2
    ty = sum(l * e[1] for l, e in zip(lam, sp._E)) / 2
    mass, m2 = Fr(0), np.zeros((2, 2))
    for i in range(-33, 34):
        for j in range(-33, 34):
            y = (tx + (i + Fr(1, 2)) * h, ty + (j + Fr(1, 2)) * h)
            b = sp.beta_k(y[0], y[1], lam)
            if b:
                mass += b * h * h
                v = np.array([float(y[0] - tx), float(y[1] - ty)])
                m2 += float(b * h * h) * np.outer(v, v)
    want = sum(float(l) ** 2 / 12 * np.outer(e, e) for l, e in zip(lam, sp._E))
    assert abs(float(mass) - 1) < 2e-3
    assert np.allclose(m2, want, atol=0.03)
