"""The pins of tests/test_oracle_pins.py and test_oracle_generator_pins.py
are sensitive: each plausible
mistake below, planted in a copy of the oracle on the CPU, makes at least
one pin fail.  A mutant is oracle.c with one exact text replacement,
compiled like the oracle and loaded in a child process through ORC_LIB."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "ltd_sign": ("s->sd[syn] -= orc_stdp_q16(c->a_minus_mv", "s->sd[syn] += orc_stdp_q16(c->a_minus_mv"),
    "ltp_lag_off_by_one": ("t - tp - d);", "t - tp - d + 1);"),
    "ltp_window_excludes_arrival_now": ("latest_spike_at_or_before(s, pre, t - d, &tp)",
                                        "latest_spike_at_or_before(s, pre, t - d - 1, &tp)"),
    "deriv_bias_dropped": ("(int64_t)*w + (int64_t)bias_q16 + (int64_t)*sd", "(int64_t)*w + (int64_t)*sd"),
    "deriv_decay_not_rounded": ("* (int64_t)decay_q16 + 32768)", "* (int64_t)decay_q16)"),
    "one_v_substep": ("for (int half = 0; half < 2; ++half) {", "for (int half = 0; half < 1; ++half) {"),
    "u_relaxes_to_c": ("    x = b * vv;                                  /* one 1 ms step of u */\n    x = x - uu;",
                       "    x = b * vv;                                  /* one 1 ms step of u */\n    x = x - c;"),
    "inhibitory_plastic_in_deriv": ("            if (!is_exc(s, p)) continue;\n            for (int64_t k = s->row_off[p]",
                                    "            for (int64_t k = s->row_off[p]"),
    "ring_member_index": ("(j - start) % 4u", "j % 4u"),
    "thalamic_wrong_draw": ("return col * c->neurons_per_col + scale_draw(r[0], c->neurons_per_col);",
                            "return col * c->neurons_per_col + scale_draw(r[1], c->neurons_per_col);"),
    "inhibitory_delay_two": ("        *delay_out = 1;\n", "        *delay_out = 2;\n"),
    "self_connection_allowed": ("if (tl >= local) tl += 1;", "(void)local;"),
    "arrival_one_step_late": ("(t + s->dly[k]) % QUEUE_SLOTS", "(t + s->dly[k] + 1) % QUEUE_SLOTS"),
    "delay_range_short": ("*delay_out = 1 + scale_draw(r[1], c->max_delay_ms);",
                          "*delay_out = 1 + scale_draw(r[1], c->max_delay_ms - 1);"),
    "current_scale": ("float cur = (float)current_q16 * 0x1p-16f;", "float cur = (float)current_q16 * 0x1p-15f;"),
    "threshold_strict": ("if (vv >= 30.0f)", "if (vv > 30.0f)"),
    "reset_double_d": ("if (vv >= 30.0f) { fired = 1; vv = c; uu = uu + d; }",
                       "if (vv >= 30.0f) { fired = 1; vv = c; uu = uu + 2.0f * d; }"),
    "current_halved_delivery": ("s->cur[post] += s->w[syn];", "s->cur[post] += s->w[syn] / 2;"),
    "fs_a_like_rs": ("else            { *a = 0.1f;", "else            { *a = 0.02f;"),
    "no_current_reset": ("s->cur[i] = 0;", ";"),
    "wmax_clamp_missing": ("if (nw > wmax_q16) nw = wmax_q16;", ";"),
    "negative_clamp_missing": ("if (nw < 0) nw = 0;", ";"),
    "period_off_by_one": ("((uint32_t)t + 1) % c->deriv_period_ms == 0", "((uint32_t)t) % c->deriv_period_ms == 0"),
    "ltd_uses_tau_plus": ('orc_stdp_q16(c->a_minus_mv, c->tau_minus_ms, t - tl)',
                          'orc_stdp_q16(c->a_minus_mv, c->tau_plus_ms, t - tl)'),
    "ltp_uses_a_minus": ('orc_stdp_q16(c->a_plus_mv, c->tau_plus_ms, t - tp - d)',
                         'orc_stdp_q16(c->a_minus_mv, c->tau_plus_ms, t - tp - d)'),
    "stdp_truncates": ("return (int32_t)llround(value);", "return (int32_t)value;"),
    "inh_targets_any": ('*target_out = col * npc + scale_draw(r[0], ne);',
                        '*target_out = col * npc + scale_draw(r[0], npc);'),
    "self_excl_strict": ("if (tl >= local) tl += 1;", "if (tl > local) tl += 1;"),
    "pct_ceil": ('uint32_t end = (uint32_t)(((uint64_t)m * acc) / 100u);',
                 'uint32_t end = (uint32_t)(((uint64_t)m * acc + 99u) / 100u);'),
    "ring2_member_order": ("{1, -1, 1, -1}", "{1, 1, -1, -1}"),
    "thal_domain0": ("draw(c, (uint32_t)t, col, 1u, k, r);", "draw(c, (uint32_t)t, col, 0u, k, r);"),
    "floor_div_truncates": ("if ((x % 65536) != 0 && x < 0) q -= 1;", ";"),
    "l_exc_not_counted": ("s->l_exc += s->in_off[post + 1] - s->in_off[post];", ";"),
    "e_exc_all": ("        s->e_exc++;\n", "        ;\n"),
    "f64_u_relax_c": ("uu = uu + a * (b * vv - uu);", "uu = uu + a * (b * vv - c);"),
    "f64_one_substep": ('for (int half = 0; half < 2; ++half)\n        vv = vv',
                        'for (int half = 0; half < 1; ++half)\n        vv = vv'),
    "wrap_no_neg": ("return r < 0 ? r + n : r;", "return r < 0 ? 0 : r;"),
    "exc_delay_zero_based": ('*delay_out = 1 + scale_draw(r[1], c->max_delay_ms);',
                             '*delay_out = scale_draw(r[1], c->max_delay_ms) + (r[1] & 1);'),
    "key_halves_swapped": ('uint32_t key[2] = {(uint32_t)(c->seed & 0xffffffffu), (uint32_t)(c->seed >> 32)};',
                           'uint32_t key[2] = {(uint32_t)(c->seed >> 32), (uint32_t)(c->seed & 0xffffffffu)};'),
    "thal_amp_once_per_col": ('for (uint32_t k = 0; k < c->thal_per_col_per_ms; ++k)\n            s->cur',
                              'for (uint32_t k = 0; k < 1; ++k)\n            s->cur'),
    "incoming_count_includes_inhibitory": (
        "if (!is_exc(s, p)) continue;\n"
        "        for (int64_t k = s->row_off[p]; k < s->row_off[p + 1]; ++k) count[",
        "for (int64_t k = s->row_off[p]; k < s->row_off[p + 1]; ++k) count["),
    # operation order of the neuron update (the bit-exact sequence)
    "f32_minus_u_plus_i_swapped": ("        x = x - uu;\n        x = x + cur;", "        x = x + cur;\n        x = x - uu;"),
    "f32_quadratic_not_horner": ("        x = 0.04f * vv;\n        x = x + 5.0f;\n        x = x * vv;",
                                 "        x = vv * vv;\n        x = 0.04f * x;\n        x = x + 5.0f * vv;"),
    # (where the factor 0.5 of the half step is applied is not observable:
    # scaling by a power of two commutes with rounding in the normal range)
    "f32_rest_constant_folded_with_u": ("        x = x + 140.0f;\n        x = x - uu;",
                                        "        x = x + (140.0f - uu);"),
    "f32_u_step_distributed": ("    x = x - uu;\n    x = a * x;\n    uu = uu + x;",
                               "    x = a * x;\n    x = x - a * uu;\n    uu = uu + x;"),
    "f64_minus_u_plus_i_swapped": ("140.0 - uu + cur)", "140.0 + cur - uu)"),
    "f64_quadratic_not_horner": ("((0.04 * vv + 5.0) * vv + 140.0", "(0.04 * (vv * vv) + 5.0 * vv + 140.0"),
}


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_mutant(workdir, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, "mutation site not unique: %s" % name
    d = workdir / name
    d.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), d / "oracle.h")
    (d / "oracle.c").write_text(text.replace(old, new))
    lib = d / "liborc.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", str(lib), str(d / "oracle.c"), "-lm"], check=True)
    env = dict(os.environ, ORC_LIB=str(lib))
    pins = [os.path.join(HERE, f) for f in ("test_oracle_generator_pins.py", "test_oracle_pins.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", *pins, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "no pin failed for mutant %s:\n%s" % (name, r.stdout[-1500:])
