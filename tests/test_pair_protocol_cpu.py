"""The exit protocol of the CTA-pair form of the persistent tensor-core
kernel, checked on a model of its barriers over many random interleavings.

In the pair form the copies of both CTAs complete on the even CTA's "full"
barrier of a stage slot, which the even CTA alone arms for the bytes of both
(arrive + expect_tx); the odd CTA's producer only waits for the slot to be
freed by the MMA completion.  Either CTA may stop issuing at any point (a
wait that ran out), and a copy may land at any time after its issue.  At the
end the even CTA settles every stage that only one CTA filled -- it arms the
ones the odd CTA filled alone and counts the bytes that were never sent --
and waits for the last phase of every slot, so that no copy can complete
towards a CTA that has left.

The model follows the mbarrier rules (a phase completes when its pending
arrival count and its transaction count are both zero; the transaction
count may go negative while arrivals are pending) and asserts what the
protocol relies on: every arrival and every landing copy acts on the phase
it was meant for, the two CTAs' stage counts differ by at most the ring
depth, and after the settlement every issued copy has landed and the last
phase of every slot has completed."""
import random

import pytest

TX = 24576          # bytes one CTA's copies bring into one stage (J tile + half the q tile)


class Barrier:
    def __init__(self):
        self.phase = 0          # completed phases
        self.pending = 1        # arrivals still expected in the current phase
        self.tx = 0             # transaction bytes still expected

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = 1

    def arrive_expect_tx(self, phase, nbytes):
        assert self.phase == phase, "arrival for phase %d while the barrier is in phase %d" % (phase, self.phase)
        assert self.pending == 1
        self.tx += nbytes
        self.pending -= 1
        self._check()

    def complete_tx(self, phase, nbytes):
        assert self.phase == phase, "bytes for phase %d while the barrier is in phase %d" % (phase, self.phase)
        self.tx -= nbytes
        self._check()


def run_once(rng, HS, npos, p_abort):
    full = [Barrier() for _ in range(HS)]
    consumed = 0                       # stages the MMA warp has consumed (frees slot k for k + HS)
    own = odd = 0                      # stages armed by the even CTA / issued by the odd CTA
    stopped = {"even": False, "odd": False, "mma": False}
    flight = []                        # copies issued and not landed: (stage k, bytes)

    def can_fill(k):                   # the slot of stage k is free once stage k - HS was consumed
        return k < HS or consumed > k - HS

    def actions():
        acts = []
        if not stopped["even"] and own < npos and can_fill(own):
            acts.append("even")
        if not stopped["odd"] and odd < npos and can_fill(odd):
            acts.append("odd")
        if not stopped["mma"] and consumed < npos and full[consumed % HS].phase > consumed // HS:
            acts.append("mma")
        if flight:
            acts.append("land")
        for who in ("even", "odd", "mma"):
            if not stopped[who] and rng.random() < p_abort:
                acts.append("stop-" + who)
        return acts

    while True:
        acts = actions()
        if not acts:
            break
        a = rng.choice(acts)
        if a == "even":
            k = own
            full[k % HS].arrive_expect_tx(k // HS, 2 * TX)
            flight.append((k, TX))
            own += 1
        elif a == "odd":
            flight.append((odd, TX))
            odd += 1
        elif a == "mma":
            consumed += 1
        elif a == "land":
            k, nbytes = flight.pop(rng.randrange(len(flight)))
            full[k % HS].complete_tx(k // HS, nbytes)
        else:
            stopped[a[5:]] = True
    # Every role has stopped or waits for ever; the bounded waits run out and
    # no copy is issued after this point.  Copies still in flight may land
    # at any time, also during the settlement.
    assert abs(own - odd) <= HS
    lo, hi = min(own, odd), max(own, odd)
    for k in range(lo, hi):
        while flight and rng.random() < 0.3:
            kk, nbytes = flight.pop(rng.randrange(len(flight)))
            full[kk % HS].complete_tx(kk // HS, nbytes)
        b = full[k % HS]
        if k >= own:
            b.arrive_expect_tx(k // HS, 2 * TX)     # filled by the odd CTA alone
        b.complete_tx(k // HS, TX)                  # the bytes never sent
    rng.shuffle(flight)
    for kk, nbytes in flight:
        full[kk % HS].complete_tx(kk // HS, nbytes)
    # the even CTA's final wait: the last phase of every slot has completed
    for k in range(max(0, hi - HS), hi):
        assert full[k % HS].phase >= k // HS + 1, "stage %d never completes" % k
    # and no slot has completed a phase nobody filled
    for s in range(HS):
        filled = [k for k in range(hi) if k % HS == s]
        assert full[s].phase == len(filled)
    return own, odd, consumed


@pytest.mark.parametrize("HS,npos", [(3, 40), (4, 64), (2, 9)])
def test_settlement_completes_every_stage_under_random_interleavings(HS, npos):
    rng = random.Random(1000 * HS + npos)
    uneven = {"even ahead": 0, "odd ahead": 0}
    for it in range(3000):
        p_abort = (0.0, 0.002, 0.02, 0.1)[it % 4]
        own, odd, _ = run_once(rng, HS, npos, p_abort)
        if own > odd:
            uneven["even ahead"] += 1
        elif odd > own:
            uneven["odd ahead"] += 1
    # both settlement branches were exercised
    assert uneven["even ahead"] > 50 and uneven["odd ahead"] > 50


def test_a_run_without_aborts_needs_no_settlement():
    rng = random.Random(7)
    for _ in range(200):
        own, odd, consumed = run_once(rng, 3, 30, 0.0)
        assert own == odd == consumed == 30
