"""The oracle's pins have teeth: plausible mistakes planted in copies of the
oracle source (compiled on the CPU, never used elsewhere) must each make at
least one pin fail.  Each mutation is a dropped term, a wrong sign, bound or
index, a transposed operand, or a reordered step."""
import os
import subprocess
import sys

import pytest

import oracle
import synth
import test_oracle_deskew as deskew
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "dbtsdf_oracle.c")

MUTATIONS = {
    "eq3_floor_not_ceil": ("int c = (int)ceil(r);", "int c = (int)floor(r);"),
    "eq3_shift_off_by_one": ("return 0xFFFFFFFFu >> (32 - c);", "return 0xFFFFFFFFu >> (31 - c);"),
    "shadow_plane_excluded": ("return dot >= 0.0;\n    double uu", "return dot > 0.0;\n    double uu"),
    "shadow_front_half": ("return dot >= 0.0;\n    double uu", "return dot <= 0.0;\n    double uu"),
    "cone_squared_norm": ("return dot >= p->shadow_cos * sqrt(r2 * uu);",
                          "return dot >= p->shadow_cos * (r2 * uu);"),
    "cone_dir_norm_dropped": ("return dot >= p->shadow_cos * sqrt(r2 * uu);",
                              "return dot >= p->shadow_cos * sqrt(r2);"),
    "cone_ignored": ("    if (p->shadow_cos == 0.0)\n        return dot >= 0.0;",
                     "    if (1)\n        return dot >= 0.0;"),
    "shadow_radius_strict": ("if (!(r2 <= p->shadow_radius * p->shadow_radius))",
                             "if (!(r2 < p->shadow_radius * p->shadow_radius))"),
    "eq6_strict_threshold": ("if (h_old < p->hit_threshold && h_new >= p->hit_threshold)\n"
                             "                        g->sign[v] = 0;",
                             "if (h_old < p->hit_threshold && h_new > p->hit_threshold)\n"
                             "                        g->sign[v] = 0;"),
    "eq5_no_saturation": ("                    if (h_new > p->hit_max)\n"
                          "                        h_new = p->hit_max;\n"
                          "                    g->hits[v] = (uint16_t)h_new;",
                          "                    g->hits[v] = (uint16_t)h_new;"),
    "pose_transposed": ("d[r] = (pose[4 * r + 0] * px + pose[4 * r + 1] * py) + pose[4 * r + 2] * pz;",
                        "d[r] = (pose[4 * 0 + r] * px + pose[4 * 1 + r] * py) + pose[4 * 2 + r] * pz;"),
    "translation_dropped": ("w[r] = d[r] + pose[4 * r + 3];", "w[r] = d[r];"),
    "boundary_off_by_one": ("if (!(q >= (double)R && q <= (double)(n[a] - 1 - R)))",
                            "if (!(q >= (double)R && q <= (double)(n[a] - R)))"),
    "last_return_kept": ("    for (int64_t i = 0; i < n; i++) {\n        if (i % ds != 0)",
                         "    for (int64_t i = n - 1; i >= 0; i--) {\n        if (i % ds != 0)"),
    "octa_fold_swapped": ("double fu = (1.0 - fabs(v)) * orc_sgn(u);", "double fu = (1.0 - fabs(u)) * orc_sgn(u);"),
    "el_edge_sign": ("return (ORC_PI * (double)k) / (double)bel - ORC_PI / 2.0;",
                     "return (ORC_PI * (double)k) / (double)bel + ORC_PI / 2.0;"),
    "az_edge_test_sign": ("ge = (cos(t) * y - sin(t) * x) >= 0.0;", "ge = (cos(t) * y + sin(t) * x) >= 0.0;"),
    "kernel_index_transposed": ("int64_t v = ((c[2] + oz) * g->ny + (c[1] + oy)) * g->nx + (c[0] + ox);",
                                "int64_t v = ((c[2] + oz) * g->ny + (c[1] + ox)) * g->nx + (c[0] + oy);"),
    "bin_from_sensor_frame": ("*bin = orc_bin(p, d[0], d[1], d[2]);", "*bin = orc_bin(p, px, py, pz);"),
    "slice_index_not_periodic": ("int64_t m = ((i % period) * (int64_t)n_poses) / period;",
                                 "int64_t m = (i * (int64_t)n_poses) / period;\n"
                                 "        if (m >= n_poses) m = n_poses - 1;"),
    "downsample_offset": ("if (i % ds != 0)\n            continue;",
                          "if (i % ds != ds - 1)\n            continue;"),
    "yaw_not_wrapped": ("        while (dpsi <= -ORC_PI)\n            dpsi += 2.0 * ORC_PI;",
                        "        while (0)\n            dpsi += 2.0 * ORC_PI;"),
    "full_interp_wrong_side": ("Q[r][c] = R0[r][0] * E[0][c] + R0[r][1] * E[1][c] + R0[r][2] * E[2][c];",
                               "Q[r][c] = E[r][0] * R0[0][c] + E[r][1] * R0[1][c] + E[r][2] * R0[2][c];"),
    "voxel_reciprocal": ("double q = floor((w[a] - g->origin[a]) / g->res);",
                         "double q = floor((w[a] - g->origin[a]) * (1.0 / g->res));"),
    "transform_fused": ("d[r] = (pose[4 * r + 0] * px + pose[4 * r + 1] * py) + pose[4 * r + 2] * pz;",
                        "d[r] = fma(pose[4 * r + 2], pz, fma(pose[4 * r + 1], py, pose[4 * r + 0] * px));"),
    "octa_reciprocal": ("    double u = dx / s;\n    double v = dy / s;",
                        "    double u = dx * (1.0 / s);\n    double v = dy * (1.0 / s);"),
    "octa_dir_not_folded": ("    if (Z < 0.0) {\n        double fu = ((double)n - fabs(V)) * orc_sgn(U);",
                            "    if (Z < -1e300) {\n        double fu = ((double)n - fabs(V)) * orc_sgn(U);"),
}


def _battery(room):
    """Run the pins against whatever oracle library is loaded; return failures."""
    orc = oracle
    checks = [
        lambda: pins.test_eq3_golden_values(orc),
        lambda: pins.test_eq3_table_closed_form(orc, 21),
        lambda: pins.test_octa_golden(orc),
        lambda: pins.test_octa_centre_round_trip(orc, 8),
        lambda: pins.test_azel_golden(orc),
        lambda: pins.test_azel_matches_atan2_asin(orc, 40, 40),
        lambda: pins.test_ball_counts_oeis(orc),
        lambda: pins.test_shadow_radius_one(orc),
        lambda: pins.test_shadow_lies_behind_surface(orc),
        lambda: pins.test_cone_exact_integer_form(orc, 1, 2),
        lambda: pins.test_cone_narrows_to_the_ray(orc),
        lambda: pins.test_single_point_worked_example(orc),
        lambda: pins.test_brute_force_tiny_grids(orc, pins.CASES[0]),
        lambda: pins.test_brute_force_tiny_grids(orc, pins.CASES[1]),
        lambda: pins.test_brute_force_tiny_grids(orc, pins.CASES[3]),
        lambda: pins.test_first_return_rule_uses_first_bin(orc),
        lambda: pins.test_border_returns_change_nothing(orc),
        lambda: pins.test_rs0_hits_count_points_per_voxel(orc, room),
        lambda: pins.test_contact_floors_follow_the_written_formulas(orc),
        lambda: deskew.test_downsampling_is_every_ds_th_return(orc, 3),
        lambda: deskew.test_one_pose_per_slice_equals_returns_one_by_one(orc),
        lambda: [deskew.test_interp_endpoints_and_rotations(orc, k, m) for k in range(4) for m in (0, 1)],
        lambda: [deskew.test_yaw_interp_turns_about_map_z_only(orc, k) for k in range(3)],
    ]
    failed = []
    for i, c in enumerate(checks):
        try:
            c()
        except (AssertionError, Exception):
            failed.append(i)
    return failed


@pytest.fixture(scope="module")
def room():
    return synth.room_scan(n_scans=1)


def test_unmutated_oracle_passes_battery(room):
    assert _battery(room) == []


_RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, synth
import test_oracle_mutations as m
oracle._lib = oracle.load({so!r})
print("FAILED", m._battery(synth.room_scan(n_scans=1)))
"""


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    """Each mutant runs the battery in its own process (a mutant that writes
    out of bounds may crash it, which also counts as caught)."""
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(src.replace(old, new, 1))
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    str(so), str(c), "-lm"], check=True)
    tests_dir = os.path.dirname(os.path.abspath(__file__))
    code = _RUNNER.format(root=os.path.dirname(tests_dir), tests=tests_dir, so=str(so))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if r.returncode < 0:
        return                                   # killed by a signal: caught
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")][-1]
    assert line != "FAILED []", f"no pin caught mutation {name}"
