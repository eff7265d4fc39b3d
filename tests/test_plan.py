"""Host-side work decomposition of the force kernels (plan_ipar / plan_jpar in
csrc/nb_internal.cuh), compiled from the same header as the library and
checked over a grid of sizes on the CPU.

Invariants: the slices cover [0, n) exactly once, slices are whole tiles,
partial sums fit the buffer whenever there is more than one slice, the item
count is i-blocks x slices, and the regime boundaries are consistent.
"""
import itertools
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include "nb_internal.cuh"
using namespace nbk;
int main() {
    int na, n, iblk, tile, slots, split; long long cap; char kind;
    while (std::scanf(" %c %d %d %d %d %d %d %lld", &kind, &na, &n, &iblk, &tile, &slots, &split, &cap) == 8) {
        if (kind == 'c') {   // slice combine: lanes per output for na outputs, n slices
            std::printf("%d 0 0 0\n", combine_lanes(na, n));
            continue;
        }
        if (kind == 'r') {   // regime for na active with jpar_max = n, small_max = iblk
            std::printf("%d 0 0 0\n", regime_of(na, n, iblk));
            continue;
        }
        if (kind == 'f') {   // whole force plan: precision = tile, split = split, slots = slots
            ForceArgs fa{};
            fa.n = n;
            fa.precision = tile;
            fa.summation = NB_SUM_COMPENSATED;
            fa.jpar_max = tile == NB_FP64 ? kJparMaxActive64 : kJparMaxActive;
            fa.small_max = tile == NB_FP64 ? 0 : kSmallMaxActive;
            fa.split = split;
            fa.slots_ipar = fa.slots_jpar = fa.slots_small = slots;
            fa.part_cap = cap;
            const ForcePlan f = make_force_plan(fa, na);
            std::printf("%d %d %d %d %d %d %d %d %d %d\n", f.regime, f.ic, f.lanes, f.p.n_iblk, f.p.S,
                        f.p.jslice, f.p.items, f.na, f.p.n_whole, f.p.a0);
            continue;
        }
        if (kind == 't' || kind == 'u') {   // i-parallel plan with the tail split allowed
            const Plan p = plan_ipar(na, n, iblk, tile, slots, split, cap, kind == 't');
            // work items in launch order: i-block, slice, j range (checked for coverage)
            long long cover = 0, bad = 0;
            for (int w = 0; w < p.items; ++w) {
                int ib, sl, j0, j1;
                ipar_item(w, p.n_iblk, p.n_whole, p.S, p.jslice, n, ib, sl, j0, j1);
                if (ib < 0 || ib >= p.n_iblk || (sl < 0) != (ib < p.n_whole || p.S == 1)) ++bad;
                if (sl >= 0 && (sl >= p.S || j0 != sl * p.jslice)) ++bad;
                cover += (long long)(j1 > j0 ? j1 - j0 : 0);
            }
            std::printf("%d %d %d %d %d %d %lld %lld\n", p.n_iblk, p.S, p.jslice, p.items, p.n_whole,
                        p.a0, cover, bad);
            continue;
        }
        Plan p = kind == 'i' ? plan_ipar(na, n, iblk, tile, slots, split, cap)
                             : plan_jpar(na, n, tile, iblk, slots, cap);
        std::printf("%d %d %d %d\n", p.n_iblk, p.S, p.jslice, p.items);
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("plan")
    src = d / "plan.cpp"
    src.write_text(SRC)
    exe = d / "plan"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_cs_0702135_gb300", "csrc"), "-I" + cuda_inc,
                    str(src), "-o", str(exe)], check=True)
    return exe


def _run(exe, cases):
    inp = "\n".join(" ".join(str(v) for v in c) for c in cases)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    return [tuple(int(v) for v in line.split()) for line in out.strip().splitlines()]


def _part_cap(n, slots, f64):
    # the context's partial buffer: 16 slots of i-blocks, four slices of all
    # n, or the j-parallel kernel's 8 slots of 4-i chunks, in 7-value records
    iblk = 64 * (1 if f64 else 4)
    return 7 * max(16 * slots * iblk, 4 * n, 8 * slots * 4)


def test_ipar_plans(planner):
    cases = []
    for na, n, (iblk, tile), slots, split in itertools.product(
            [1, 17, 64, 191, 256, 1000, 4096, 65536, 1 << 20], [2, 130, 4099, 65536, 1 << 20],
            [(256, 64), (64, 64), (128, 128)], [152, 608, 2432], [0, 1, 7]):
        if na > n:
            continue
        cap = 7 * max(16 * slots * iblk, 4 * n)
        cases.append(("i", na, n, iblk, tile, slots, split, cap))
    for c, (nib, S, js, items) in zip(cases, _run(planner, cases)):
        _, na, n, iblk, tile, slots, split, cap = c
        assert nib == -(-na // iblk)
        assert S >= 1 and js % tile == 0 and js > 0
        assert (S - 1) * js < n <= S * js, c
        assert items == nib * S
        if S > 1:
            assert S * 7 * na <= cap, c
        if split:
            assert S <= split
        # enough work items to fill the GPU whenever the slices allow it: the
        # plan aims at two per resident CTA; rounding slices up to whole tiles
        # can at most halve the slice count, so at least one full wave remains
        if split == 0 and nib < 2 * slots and -(-n // (2 * tile)) >= 2 * slots:
            assert items >= slots, c


def test_jpar_plans(planner):
    cases = []
    for na, n, slots, ic in itertools.product([1, 2, 4, 5, 16, 32, 33], [2, 300, 65536, 1 << 20],
                                              [152, 304], [1, 4]):
        if na > n:
            continue
        cap = 7 * 8 * slots * 4
        cases.append(("j", na, n, ic, 256, slots, 0, cap))
    for c, (nch, S, js, items) in zip(cases, _run(planner, cases)):
        _, na, n, ic, nt, slots, _, cap = c
        assert nch == -(-na // ic)
        assert (S - 1) * js < n <= S * js and js % nt == 0
        # partials are stored per chunk slot: ic values of 7 components per slice
        assert S * 7 * nch * ic <= cap
        assert items == nch * S
        assert S == 1 or js >= 8 * nt
        # a lone particle on 2^20 bodies fills two waves, or one when the
        # slices of two would be too short, never one and a fraction
        # (rounding the slices to whole tiles loses a few percent)
        if na == 1 and n == 1 << 20:
            waves = 2 if 2 * slots * 8 * nt <= n else 1
            assert 0.9 * waves * slots <= items <= waves * slots, c


def test_combine_lanes(planner):
    cases = [("c", na, S, 0, 0, 0, 0, 0) for na in (1, 2, 7, 33, 300, 1820, 4096, 65536, 1 << 20)
             for S in (1, 2, 3, 8, 9, 76, 512, 2432)]
    for c, (T, _, _, _) in zip(cases, _run(planner, cases)):
        _, na, S = c[:3]
        assert T in (1, 2, 4, 8, 16, 32), c
        assert T == 1 or T <= S, c
        # doubling T would pass 2^18 threads or S, or T is already 32
        assert T == 32 or 2 * T > S or T * 7 * na >= 1 << 18, c


def test_regimes(planner):
    # automatic mode: j-parallel up to 96, then the one-i-per-thread kernel
    # whenever its 64-i padding is at most 3/4 of the 256-i padding
    cases = [("r", na, 96, 1024, 0, 0, 0, 0) for na in range(1, 1500)]
    got = {c[1]: r[0] for c, r in zip(cases, _run(planner, cases))}
    small = {na for na in range(1, 1500) if 96 < na <= 192 or 256 < na <= 384 or 512 < na <= 576}
    for na, reg in got.items():
        want = 0 if na <= 96 else (1 if na in small else 2)
        assert reg == want, (na, reg)
    # small_max <= jpar_max disables the small-block kernel; jpar_max = 0 the j-parallel one
    cases = [("r", na, 0, 0, 0, 0, 0, 0) for na in (1, 100, 300)]
    assert [r[0] for r in _run(planner, cases)] == [2, 2, 2]


def test_force_plans(planner):
    # The plan a force launch runs with, for both precisions: the serving
    # kernel, i per pass (one for DS blocks of one or two), the slice partials
    # within the buffer, the combine's lanes, and the slices covering all j.
    cases = []
    for na, n, slots, prec, split in itertools.product(
            [1, 2, 3, 5, 32, 33, 96, 97, 192, 193, 300, 513, 600, 4096, 65536],
            [100, 3001, 65536, 1 << 20], [608, 1216, 2432], [0, 1], [0, 3]):
        if na > n:
            continue
        cases.append(("f", na, n, 0, prec, slots, split, _part_cap(n, slots, prec == 1)))
    for c, out in zip(cases, _run(planner, cases)):
        _, na, n, _, prec, slots, split, cap = c
        regime, ic, lanes, nib, S, js, items, fna, n_whole, a0 = out
        assert fna == na
        jmax = 32 if prec == 1 else 96
        if na <= jmax:
            assert regime == 0, c
            assert ic == (1 if prec == 0 and na <= 2 else 4), c
            assert nib * ic * 7 * S <= cap, c          # j-parallel partials per chunk slot
        else:
            assert regime in (1, 2) and (prec == 0 or regime == 2), c
            assert ic == 0
            assert S == 1 or S * 7 * (na - a0) <= cap, c
            if split:
                assert S <= split and n_whole == 0
        assert (S - 1) * js < n <= S * js and items == n_whole + (nib - n_whole) * S, c
        assert n_whole == 0 or (regime != 0 and n_whole % slots == 0 and a0 < na), c
        assert lanes in (1, 2, 4, 8, 16, 32) and (lanes == 1 or lanes <= S), c


def _wave_cost(items, slots, length):
    return -(-items // slots) * (length + 64)


def test_tail_split_plans(planner):
    # With at least one full wave of i-blocks the blocks of the full waves may
    # run whole and only the remainder be sliced.  Every (i-block, j) pair is
    # covered exactly once (the j lengths of all items add up to n per
    # i-block), whole blocks come first and are multiples of the resident
    # slots, the sliced blocks' partials fit the buffer, and the split is
    # taken only when its wave cost is below the uniform plan's.
    cases = []
    for na, n, slots in itertools.product(
            [1000, 155648, 155649, 200000, 262144, 300001, 1 << 20, (1 << 20) - 3],
            [262144, 300001, 1 << 20], [152, 608, 1216]):
        if na > n:
            continue
        cap = 7 * max(16 * slots * 256, 4 * n)
        cases.append(("t", na, n, 256, 128, slots, 0, cap))
        cases.append(("u", na, n, 256, 128, slots, 0, cap))
    out = _run(planner, cases)
    split_seen = 0
    for k in range(0, len(cases), 2):
        c, t, u = cases[k], out[k], out[k + 1]
        _, na, n, iblk, tile, slots, _, cap = c
        nib, S, js, items, n_whole, a0, cover, bad = t
        assert bad == 0, c
        assert cover == nib * n, c
        assert (S - 1) * js < n <= S * js and js % tile == 0, c
        assert items == n_whole + (nib - n_whole) * S, c
        unib, uS, ujs, uitems, un_whole, ua0, ucover, ubad = u
        assert un_whole == 0 and ua0 == 0 and ubad == 0 and ucover == unib * n
        if n_whole == 0:
            assert (S, js, items) == (uS, ujs, uitems), c
            continue
        split_seen += 1
        rem = nib - n_whole
        assert nib >= slots and n_whole % slots == 0 and 0 < rem < slots, c
        assert a0 == n_whole * iblk and S >= 2, c
        assert S * 7 * (na - a0) <= cap, c
        c_split = _wave_cost(n_whole, slots, n) + _wave_cost(rem * S, slots, js)
        assert c_split < _wave_cost(uitems, slots, ujs), c
    assert split_seen >= 10
    # the benchmark's sweep: 2^20 bodies, 608 resident CTAs of 256 i
    (nib, S, js, items, n_whole, a0, cover, bad), = _run(
        planner, [("t", 1 << 20, 1 << 20, 256, 128, 608, 0, 7 * 16 * 608 * 256)])
    assert (nib, n_whole, S) == (4096, 3648, 19) and items == 3648 + 448 * 19
    assert items % 608 == 0


def test_tail_split_plans_random(planner):
    # Seeded random block sizes, body counts and resident slots around and
    # above one full wave of i-blocks, for both i-block sizes (four i per
    # thread, one i per thread): the same invariants as above on every case.
    import random
    r = random.Random(23)
    cases = []
    for _ in range(3000):
        iblk = r.choice([256, 64])
        slots = r.choice([152, 304, 608, 1216, 2432])
        n = r.randint(iblk * slots // 2, 3 << 20)
        lo = min(n, max(1, iblk * slots - 5000))
        na = r.randint(lo, n) if r.random() < 0.7 else r.randint(1, n)
        cap = 7 * max(16 * slots * iblk, 4 * n)
        cases.append(("t", na, n, iblk, 128, slots, 0, cap))
    out = _run(planner, cases)
    seen = 0
    for c, (nib, S, js, items, n_whole, a0, cover, bad) in zip(cases, out):
        _, na, n, iblk, tile, slots, _, cap = c
        assert bad == 0 and cover == nib * n, c
        assert (S - 1) * js < n <= S * js and js % tile == 0, c
        assert items == n_whole + (nib - n_whole) * S, c
        if n_whole:
            seen += 1
            rem = nib - n_whole
            assert n_whole % slots == 0 and 0 < rem < slots and a0 == n_whole * iblk, c
            assert S >= 2 and S * 7 * (na - a0) <= cap, c
        elif S > 1:
            assert S * 7 * na <= cap, c
    assert seen > 500
