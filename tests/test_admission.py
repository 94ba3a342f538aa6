"""The serving loop's admission rule (first fitting job, then continuous
batching of later small jobs of the same mode and algorithm), driven on the
host through tests/admission_driver.cpp."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2103_05162_gb300", "csrc")


@pytest.fixture(scope="module")
def driver():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    bdir = os.path.join(HERE, "_build")  # git-ignored
    os.makedirs(bdir, exist_ok=True)
    out = os.path.join(bdir, "admission_driver")
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, os.path.join(HERE, "admission_driver.cpp"),
                    "-o", out], check=True)
    return out


def pick(driver, jobs, budget=1000, used=0, job_points=100, batch_points=1000, batch_jobs=8, per_point=1,
         per_job=0):
    """jobs: (n, mode, algo, bytes). Returns (bytes, chosen, left)."""
    lines = [f"{budget} {used} {job_points} {batch_points} {batch_jobs} {per_point} {per_job} {len(jobs)}"]
    lines += [f"{n} {m} {a} {b}" for n, m, a, b in jobs]
    r = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    out = r.stdout.split("\n")
    return int(out[0]), [int(x) for x in out[1].split()], [int(x) for x in out[2].split()]


def test_first_fitting_job_is_taken(driver):
    # job 0 does not fit next to 600 used bytes, job 1 does
    b, chosen, left = pick(driver, [(500, 0, 0, 500), (300, 0, 0, 300), (50, 0, 0, 50)], used=600,
                           job_points=0)
    assert (b, chosen, left) == (300, [1], [0, 2])


def test_nothing_fits(driver):
    b, chosen, left = pick(driver, [(500, 0, 0, 500), (400, 0, 0, 400)], used=700)
    assert (b, chosen, left) == (0, [], [0, 1])


def test_empty_queue(driver):
    assert pick(driver, []) == (0, [], [])


def test_small_jobs_merge_in_queue_order(driver):
    jobs = [(10, 0, 1, 40), (200, 0, 1, 400), (20, 0, 1, 40), (30, 1, 1, 40), (40, 0, 0, 40), (50, 0, 1, 40)]
    b, chosen, left = pick(driver, jobs)
    # large job 1, other mode (3) and other algorithm (4) stay queued
    assert chosen == [0, 2, 5] and left == [1, 3, 4]
    assert b == 10 + 20 + 50  # the batch model: 1 byte per point


def test_large_head_runs_alone(driver):
    jobs = [(500, 0, 1, 500), (10, 0, 1, 10), (10, 0, 1, 10)]
    assert pick(driver, jobs) == (500, [0], [1, 2])


def test_merging_off(driver):
    jobs = [(10, 0, 1, 10), (10, 0, 1, 10)]
    assert pick(driver, jobs, job_points=0) == (10, [0], [1])


def test_automatic_choice_jobs_never_merge(driver):
    jobs = [(10, 0, 2, 10), (10, 0, 2, 10), (10, 0, 1, 10)]
    assert pick(driver, jobs) == (10, [0], [1, 2])
    jobs = [(10, 0, 1, 10), (10, 0, 2, 10), (10, 0, 1, 10)]
    b, chosen, left = pick(driver, jobs)
    assert chosen == [0, 2] and left == [1]


def test_batch_point_and_job_limits(driver):
    jobs = [(60, 0, 0, 60)] * 6
    b, chosen, left = pick(driver, jobs, batch_points=150)
    assert chosen == [0, 1] and left == [2, 3, 4, 5] and b == 120
    b, chosen, left = pick(driver, jobs, batch_points=10_000, batch_jobs=3)
    assert chosen == [0, 1, 2] and left == [3, 4, 5]


def test_batch_respects_budget(driver):
    # each join adds 100 bytes per job to the batch workspace; budget stops at 3 jobs
    jobs = [(10, 0, 0, 10)] * 5
    b, chosen, left = pick(driver, jobs, budget=350, per_point=0, per_job=100)
    assert chosen == [0, 1, 2] and left == [3, 4] and b == 300


def test_a_job_that_would_overflow_is_skipped_not_blocking(driver):
    # job 1 would push the batch past batch_points; job 2 still joins
    jobs = [(50, 0, 0, 50), (90, 0, 0, 90), (40, 0, 0, 40)]
    b, chosen, left = pick(driver, jobs, batch_points=100)
    assert chosen == [0, 2] and left == [1] and b == 90
