/*
 * toy_pipeline.c -- the project's small out-of-order CPU timing model that
 * labels synthetic traces for training (a stand-in for the gem5 timestamps of
 * Sec. 2.4; it is an input generator, not part of SimNet's method).
 *
 * Machine: fetch in order, up to 4 per cycle; a 64-entry reorder buffer
 * (instruction i is fetched no earlier than the commit of i-64); after a
 * mispredicted branch the next fetch waits until the branch completes plus 15
 * cycles.  Issue out of order, at most 4 per cycle, no earlier than fetch + 1
 * and once the last writers of both source registers have completed (greedy
 * in program order: the earliest cycle with a free issue slot).  Latency:
 * loads 1 + (opcode mod 4) + {4, 14, 200} by cache level; stores and branches
 * 1; others 1 + (opcode mod 4).  Commit in order, up to 4 per cycle, no
 * earlier than completion.
 *
 * Labels: F_i = fetch_i - fetch_{i-1} (F_0 = fetch_0 = 0), E_i = complete_i -
 * fetch_i, both clamped to 255.  Context of i: instructions j < i still
 * uncommitted when i-1 was fetched (commit_j > fetch_{i-1}); since commit is
 * in order this is the range [ctx_begin_i, i).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FETCH_W 4
#define ISSUE_W 4
#define COMMIT_W 4
#define ROB 64
#define MISPREDICT_PENALTY 15
#define SLOTS (1 << 20)   /* issue-slot table indexed by cycle mod SLOTS */

static int64_t lat_of(uint32_t r)
{
    int op = r & 31, ld = (r >> 20) & 1, st = (r >> 21) & 1, br = (r >> 22) & 1, lvl = (r >> 23) & 3;
    static const int64_t add[4] = {4, 14, 200, 200};
    if (ld) return 1 + (op % 4) + add[lvl];
    if (st || br) return 1;
    return 1 + (op % 4);
}

/* Returns 0, or -1 on allocation failure.  All outputs have n entries. */
int toy_pipeline(const uint32_t *rec, int64_t n, int64_t *fetch, int64_t *complete, int64_t *commit,
                 uint8_t *F, uint8_t *E, int64_t *ctx_begin)
{
    int64_t *slot_cycle = (int64_t *)malloc(sizeof(int64_t) * SLOTS);
    int32_t *slot_used = (int32_t *)malloc(sizeof(int32_t) * SLOTS);
    if (!slot_cycle || !slot_used) { free(slot_cycle); free(slot_used); return -1; }
    for (int64_t s = 0; s < SLOTS; s++) slot_cycle[s] = -1;
    int64_t writer_done[32];
    for (int k = 0; k < 32; k++) writer_done[k] = 0;
    int64_t prev_fetch = 0, redirect = 0, prev_commit = 0, j0 = 0;
    int fetched_in_cycle = 0, committed_in_cycle = 0;
    for (int64_t i = 0; i < n; i++) {
        const uint32_t r = rec[i];
        /* fetch */
        int64_t f = prev_fetch;
        if (i >= ROB && commit[i - ROB] > f) f = commit[i - ROB];
        if (redirect > f) f = redirect;
        if (i > 0 && f == prev_fetch && fetched_in_cycle >= FETCH_W) f++;
        fetched_in_cycle = (i > 0 && f == prev_fetch) ? fetched_in_cycle + 1 : 1;
        /* issue */
        int64_t ready = f + 1;
        int s0 = (r >> 5) & 31, s1 = (r >> 10) & 31, d = (r >> 15) & 31;
        if (writer_done[s0] > ready) ready = writer_done[s0];
        if (writer_done[s1] > ready) ready = writer_done[s1];
        int64_t c = ready;
        for (;;) {
            int64_t s = c & (SLOTS - 1);
            if (slot_cycle[s] != c) { slot_cycle[s] = c; slot_used[s] = 0; }
            if (slot_used[s] < ISSUE_W) { slot_used[s]++; break; }
            c++;
        }
        const int64_t done = c + lat_of(r);
        writer_done[d] = done;
        /* commit */
        int64_t cm = done > prev_commit ? done : prev_commit;
        if (i > 0 && cm == prev_commit && committed_in_cycle >= COMMIT_W) cm++;
        committed_in_cycle = (i > 0 && cm == prev_commit) ? committed_in_cycle + 1 : 1;
        /* branch redirect */
        if (((r >> 22) & 1) && ((r >> 25) & 1)) redirect = done + MISPREDICT_PENALTY;
        /* context of i: uncommitted at the previous fetch */
        const int64_t now = i > 0 ? fetch[i - 1] : 0;
        while (j0 < i && commit[j0] <= now) j0++;
        ctx_begin[i] = j0;
        fetch[i] = f;
        complete[i] = done;
        commit[i] = cm;
        const int64_t fl = f - (i > 0 ? prev_fetch : 0), el = done - f;
        F[i] = (uint8_t)(fl > 255 ? 255 : fl);
        E[i] = (uint8_t)(el > 255 ? 255 : el);
        prev_fetch = f;
        prev_commit = cm;
    }
    free(slot_cycle);
    free(slot_used);
    return 0;
}
